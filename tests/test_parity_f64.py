"""GPU parity of the FP64 forms against the oracle (element by element,
normwise relative error <= 1e-12 per output; bitwise for integer-valued
inputs, whose partial sums are all exact).  Shapes span several tiles of
every kernel, ragged edges, odd and padded leading dimensions, and the
empty cases."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from f64_cases import MATRIX_RUNNERS, VECTOR_RUNNERS, run_atax, run_gemver
from gpu_util import TOL64, Out, dev, p, relerr, sync, ws

pytestmark = pytest.mark.gpu

# (m, n, lda): one row/column, ragged, padded (lda > m, odd and even),
# tall, wide, several 2048-row chunks, and the empty cases.
SHAPES = [(1, 1, 1), (2, 3, 2), (3, 2, 4), (7, 31, 7), (33, 127, 33), (129, 1000, 131),
          (1000, 129, 1000), (2048, 2048, 2048), (2500, 700, 2503), (4100, 37, 4102),
          (37, 5000, 40), (5000, 300, 5000), (0, 5, 1), (5, 0, 5), (0, 0, 1)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def _check(res, tol=TOL64, exact=False):
    for name, (g, o) in res.items():
        if exact:
            assert np.array_equal(np.asarray(g, np.float64), np.asarray(o, np.float64)), name
        else:
            e = relerr(g, o)
            assert e <= tol, "%s: normwise error %.3e" % (name, e)


@pytest.mark.parametrize("form", ["fused", "unfused"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_matrix_kernel(kernel, shape, form):
    m, n, lda = shape
    _check(MATRIX_RUNNERS[kernel](m, n, max(lda, 1), synth.KIND_UNIFORM, form=form))


@pytest.mark.parametrize("form", ["fused", "unfused"])
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_matrix_kernel_integer_exact(kernel, form):
    # Integer inputs and scalars that keep every product and partial sum an
    # exact FP64 integer (|sums| < 2^53), so any summation order is exact.
    scal = {"bicgk": {}, "atax": {"beta": 2.0}, "gemver": {"alpha": 2.0, "beta": -3.0},
            "gesummv": {"alpha": 2.0, "beta": -1.0}, "dgemv": {"alpha": 3.0, "beta": -2.0},
            "dgemvt": {"alpha": -1.0, "beta": 2.0}}[kernel]
    _check(MATRIX_RUNNERS[kernel](300, 517, 302, synth.KIND_INTEGER, seed=4, form=form, **scal),
           exact=True)


@pytest.mark.parametrize("form", ["fused", "unfused"])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 1001, 65537, 1 << 20])
@pytest.mark.parametrize("kernel", sorted(VECTOR_RUNNERS))
def test_vector_kernel(kernel, n, form):
    _check(VECTOR_RUNNERS[kernel](n, synth.KIND_UNIFORM, form=form))


@pytest.mark.parametrize("kernel", sorted(VECTOR_RUNNERS))
def test_vector_kernel_integer_exact(kernel):
    _check(VECTOR_RUNNERS[kernel](100003, synth.KIND_INTEGER, seed=5), exact=True)


@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS) + sorted(VECTOR_RUNNERS))
def test_deterministic(kernel):
    if kernel in MATRIX_RUNNERS:
        a = MATRIX_RUNNERS[kernel](3001, 1777, 3001, synth.KIND_UNIFORM, seed=9)
        b = MATRIX_RUNNERS[kernel](3001, 1777, 3001, synth.KIND_UNIFORM, seed=9)
    else:
        a = VECTOR_RUNNERS[kernel](300007, synth.KIND_UNIFORM, seed=9)
        b = VECTOR_RUNNERS[kernel](300007, synth.KIND_UNIFORM, seed=9)
    for k in a:
        assert np.array_equal(a[k][0], b[k][0], equal_nan=True), k


def test_fused_unfused_bitwise_where_the_arithmetic_is_identical():
    # GEMVER's B is formed by the same two fused multiply-adds in both forms;
    # x and w are sums in a fixed order that differs between the forms (the
    # fused form's one-launch kernel sums whole columns and rows, the unfused
    # form adds panel partials), so they agree to rounding.  The vector
    # kernels perform the same operations in the same order.
    a = run_gemver(700, 333, 701, synth.KIND_UNIFORM, form="fused")
    b = run_gemver(700, 333, 701, synth.KIND_UNIFORM, form="unfused")
    assert np.array_equal(a["B"][0], b["B"][0])
    for k in ("x", "w"):
        assert relerr(a[k][0], b[k][0]) < TOL64, k
    for kern in ("vadd", "waxpby", "axpydot"):
        a = VECTOR_RUNNERS[kern](100001, synth.KIND_UNIFORM, form="fused")
        b = VECTOR_RUNNERS[kern](100001, synth.KIND_UNIFORM, form="unfused")
        for k in a:
            assert np.array_equal(a[k][0], b[k][0]), (kern, k)


def test_in_place_forms():
    m, n = 900, 611
    ids = synth.GEMVER_IDS
    A = synth.matrix(2, ids["A"], m, n)
    vecs = [synth.vector(2, ids[k], m if k in ("u1", "u2", "y") else n)
            for k in ("u1", "v1", "u2", "v2", "y", "z")]
    Bo, xo, wo = O.gemver(m, n, 1.5, 1.2, A, *vecs)
    dA = dev(A)
    d = [dev(v) for v in vecs]
    w = Out(m)
    wk, nb = ws("gemver", 0, m, n)
    # B written over A, x written over z
    bto.bto_gemver(m, n, 1.5, 1.2, p(dA), m, *[p(t) for t in d], p(dA), m, p(d[5]), w.ptr(),
                   p(wk), nb, None)
    sync()
    assert relerr(dA.cpu().numpy().reshape(n, m).T, Bo) < 1e-15
    assert relerr(d[5].cpu().numpy(), xo) < TOL64 and relerr(w.host(), wo) < TOL64
    # AXPYDOT with z == w
    nn = 70001
    wv, vv, uv = (synth.vector(3, k, nn) for k in range(3))
    zo, ro = O.axpydot(nn, 0.5, wv, vv, uv)
    dw, dv, du = dev(wv), dev(vv), dev(uv)
    r = Out(1)
    wk, nb = ws("axpydot", 0, 0, nn)
    bto.bto_axpydot(nn, 0.5, p(dw), p(dv), p(du), p(dw), r.ptr(), p(wk), nb, None)
    sync()
    assert relerr(dw.cpu().numpy(), zo) < 1e-15 and relerr(r.host(), [ro]) < TOL64
    # DGEMV with z == y
    A = synth.matrix(3, 0, 500, 400)
    xv, yv = synth.vector(3, 1, 400), synth.vector(3, 2, 500)
    zo = O.dgemv(500, 400, 2.0, A, xv, -1.0, yv)
    dA, dx, dy = dev(A), dev(xv), dev(yv)
    wk, nb = ws("dgemv", 0, 500, 400)
    bto.bto_dgemv(500, 400, 2.0, p(dA), 500, p(dx), -1.0, p(dy), p(dy), p(wk), nb, None)
    sync()
    assert relerr(dy.cpu().numpy(), zo) < TOL64


def test_nan_propagates_with_zero_beta():
    m, n = 64, 48
    A = synth.matrix(4, 0, m, n)
    xv = synth.vector(4, 1, n)
    yv = synth.vector(4, 2, m)
    yv[5] = np.nan
    for f in (bto.bto_dgemv, bto.bto_unfused_dgemv):
        z = Out(m)
        wk, nb = ws("dgemv", 0 if f is bto.bto_dgemv else 1, m, n)
        f(m, n, 1.0, dev(A), m, dev(xv), 0.0, dev(yv), z.ptr(), p(wk), nb, None)
        sync()
        zh = z.host()
        assert np.isnan(zh[5]) and np.all(np.isfinite(np.delete(zh, 5)))


def test_padding_rows_are_never_read():
    # Rows m..lda-1 hold NaN (synth pads with NaN); any read would poison results.
    for kern in sorted(MATRIX_RUNNERS):
        res = MATRIX_RUNNERS[kern](333, 257, 340, synth.KIND_UNIFORM)
        for k, (g, o) in res.items():
            assert np.all(np.isfinite(g)), (kern, k)


def test_atax_bounded_wait_times_out_and_context_survives():
    m, n = 4096, 3000
    A = synth.matrix(6, 0, m, n)
    xv = synth.vector(6, 1, n)
    dA, dx = dev(A), dev(xv)
    y = Out(n)
    wk, nb = ws("atax", 0, m, n)
    bto.bto_debug_atax_stall(m, n, 1.0, p(dA), m, p(dx), y.ptr(), p(wk), nb, 3, 50, None)
    assert bto.bto_device_status(p(wk)) == bto.BTO_ERR_TIMEOUT
    # The context is still usable and a normal call succeeds afterwards.
    bto.bto_atax(m, n, 1.0, p(dA), m, p(dx), y.ptr(), p(wk), nb, None)
    assert bto.bto_device_status(p(wk)) == 0
    assert relerr(y.host(), O.atax(m, n, 1.0, A, xv)) < TOL64


def _gemver_inputs(m, n, seed):
    A = synth.matrix(seed, 0, m, n)
    vec = {k: synth.vector(seed, i + 1, m if k in ("u1", "u2", "y") else n)
           for i, k in enumerate(("u1", "v1", "u2", "v2", "y", "z"))}
    return A, vec


def test_gemver_one_launch_matches_two_pass_and_oracle():
    """At n = 2048 bto_gemver runs both passes in one cooperative launch; with a
    schedule override it runs the panel engine's two passes.  Both match the
    oracle, B is the same bits (the same two FMAs per element), also in place."""
    m, n = 2048, 2048
    A, v = _gemver_inputs(m, n, 31)
    d = {k: dev(x) for k, x in v.items()}
    rB, rx, rw = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"])
    res = []
    for override in (False, True):
        if override:
            bto.bto_schedule_set(bto.OPS["gemver"], 0, 64, 2)
        try:
            dA = dev(A)
            B = torch.empty(m * n, dtype=torch.float64, device="cuda")
            x, w = Out(n), Out(m)
            wk, nb = ws("gemver", 0, m, n)
            bto.bto_gemver(m, n, 1.5, 1.2, p(dA), m, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]), p(d["y"]),
                           p(d["z"]), p(B), m, x.ptr(), w.ptr(), p(wk), nb, None)
            if not override:     # the one-launch form writes the status word (the panel engine has no waits)
                assert bto.bto_device_status(p(wk)) == 0
            gB = B.cpu().numpy()
            assert relerr(gB, np.asarray(rB).ravel(order="F")) < TOL64
            assert relerr(x.host(), rx) < TOL64 and relerr(w.host(), rw) < TOL64
            # in place: B over A
            bto.bto_gemver(m, n, 1.5, 1.2, p(dA), m, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]), p(d["y"]),
                           p(d["z"]), p(dA), m, x.ptr(), w.ptr(), p(wk), nb, None)
            assert np.array_equal(dA.cpu().numpy(), gB)
            assert relerr(w.host(), rw) < TOL64
            res.append(gB)
        finally:
            bto.bto_schedule_set(bto.OPS["gemver"], 0, 0, 0)
    assert np.array_equal(res[0], res[1])
    # bitwise reproducible
    x2, w2 = Out(n), Out(m)
    B2 = torch.empty(m * n, dtype=torch.float64, device="cuda")
    wk, nb = ws("gemver", 0, m, n)
    for _ in range(2):
        bto.bto_gemver(m, n, 1.5, 1.2, p(dev(A)), m, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]), p(d["y"]),
                       p(d["z"]), p(B2), m, x2.ptr(), w2.ptr(), p(wk), nb, None)
        res.append((x2.host(), w2.host()))
    assert np.array_equal(res[2][0], res[3][0]) and np.array_equal(res[2][1], res[3][1])


@pytest.mark.parametrize("plant", ["tiny_A", "huge_A", "tiny_y", "huge_z", "nan_A", "inf_v1"])
def test_gemver_one_launch_range_fallbacks(plant):
    """The one-launch form sums in double-float only for operands in
    [2^-40, 2^40]; planted values outside send a column of x, or 8 rows of w,
    to FP64.  Results match the oracle (non-finite where it is)."""
    m, n = 300, 257
    A, v = _gemver_inputs(m, n, 33)
    if plant == "tiny_A":
        A[5, 7] = 1e-30; A[100, 200] = -3e-20
    elif plant == "huge_A":
        A[17, 3] = 1e30; A[299, 256] = -2e15
    elif plant == "tiny_y":
        v["y"][9] = 1e-25
    elif plant == "huge_z":
        v["z"][11] = 1e20                       # x_11 huge: every row of w in FP64
    elif plant == "nan_A":
        A[40, 50] = np.nan
    else:
        v["v1"][60] = np.inf
    d = {k: dev(x) for k, x in v.items()}
    B = torch.empty(m * n, dtype=torch.float64, device="cuda")
    x, w = Out(n), Out(m)
    wk, nb = ws("gemver", 0, m, n)
    bto.bto_gemver(m, n, 1.5, 1.2, p(dev(A)), m, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]), p(d["y"]),
                   p(d["z"]), p(B), m, x.ptr(), w.ptr(), p(wk), nb, None)
    assert bto.bto_device_status(p(wk)) == 0
    rB, rx, rw = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"])
    for g, o in ((B.cpu().numpy(), np.asarray(rB).ravel(order="F")), (x.host(), rx), (w.host(), rw)):
        fin = np.isfinite(o)
        assert np.array_equal(np.isfinite(g), fin)
        if fin.any():
            assert relerr(g[fin], o[fin]) < TOL64


def test_gemver_grid_barrier_times_out_and_context_survives():
    m, n = 2048, 2048
    A, v = _gemver_inputs(m, n, 32)
    d = {k: dev(x) for k, x in v.items()}
    dA = dev(A)
    B = torch.empty(m * n, dtype=torch.float64, device="cuda")
    x, w = Out(n), Out(m)
    wk, nb = ws("gemver", 0, m, n)
    args = (m, n, 1.5, 1.2, p(dA), m, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]), p(d["y"]), p(d["z"]),
            p(B), m, x.ptr(), w.ptr(), p(wk), nb)
    bto.bto_debug_gemver_stall(*args, 5, 50, None)
    assert bto.bto_device_status(p(wk)) == bto.BTO_ERR_TIMEOUT
    rB, rx, rw = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"])
    assert relerr(x.host(), rx) < TOL64           # pass 1 completed before the barrier
    # no stall: the same form runs to the end; then the ordinary call
    bto.bto_debug_gemver_stall(*args, -1, 50, None)
    assert bto.bto_device_status(p(wk)) == 0
    assert relerr(w.host(), rw) < TOL64
    bto.bto_gemver(*args, None)
    assert bto.bto_device_status(p(wk)) == 0
    assert relerr(w.host(), rw) < TOL64


def test_workspace_too_small_is_rejected():
    m, n = 100, 100
    A = dev(synth.matrix(1, 0, m, n))
    v = dev(synth.vector(1, 1, n))
    q, s = Out(m), Out(n)
    wk, nb = ws("bicgk", 0, m, n)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk(m, n, p(A), m, p(v), p(v), q.ptr(), s.ptr(), p(wk), nb - 8, None)
    assert e.value.status == bto.BTO_ERR_WORKSPACE and e.value.arg == 9
