"""GPU parity of the double-float forms of the FP64 matrix sequences
(bto_*_df and bto_unfused_*_df) against the FP64 oracle.

- Normwise relative error <= 1e-12 per output (the FP64 contract) over
  shapes that span several 16-column units and 256-row chunks, ragged
  edges, several row blocks, the widest panels, and the empty cases; the
  same inputs give <= 1e-13 at n = 2048, a guard well above the form's
  47-bit arithmetic (about 1e-14) and far below what a dropped cross term
  or error term would leave (about 1e-8).
- Integer-valued inputs: exact (every product and partial sum is an exact
  FP32 double-float value), so bitwise equal to the oracle.
- FP32's range: elements of 2^128 or more, Inf and NaN, and products or
  sums that overflow FP32, take the FP64 recomputation; zeros, tiny and
  large-but-representable elements, subnormals and extreme vector elements
  stay on the double-float path.  Results match the oracle, NaN and Inf
  where it has them.
- Layouts the tensor-map copies cannot take (odd leading dimension) run the
  FP64 form: bitwise equal to it.
- GEMVER with B written over A, with and without out-of-range elements.
- Determinism and the device status word."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from f64_cases import MATRIX_RUNNERS, entry
from gpu_util import TOL64, Out, dev, p, relerr, sync, ws

pytestmark = pytest.mark.gpu

DF_FORMS = ["df", "df_unfused"]

# (m, n, lda), even leading dimensions (the double-float sweep's layout):
# single element, ragged rows and columns around the 256-row chunk and the
# 16-column unit, several row blocks (narrow matrices), the widest panels
# (n > 152 x 512), and the empty cases.
SHAPES = [(1, 1, 2), (2, 3, 2), (3, 2, 4), (7, 31, 8), (33, 127, 34), (129, 1000, 130),
          (1000, 129, 1000), (255, 17, 256), (257, 33, 258), (2048, 2048, 2048), (2500, 700, 2502),
          (4100, 37, 4102), (37, 5000, 40), (5000, 300, 5000), (300, 9000, 300), (64, 100000, 64),
          (0, 5, 2), (5, 0, 6), (0, 0, 2)]


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


@pytest.mark.parametrize("form", DF_FORMS)
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_df_matrix_kernel(kernel, shape, form):
    m, n, lda = shape
    res = MATRIX_RUNNERS[kernel](m, n, lda, synth.KIND_UNIFORM, form=form)
    if kernel == "gemver":
        # B: formed by FP64 FMAs (the FP64 form's B), a few ulps from the
        # oracle's twice-rounded sums.
        g, o = res.pop("B")
        assert relerr(g, o) <= 1e-15
    _check(res)


@pytest.mark.parametrize("form", DF_FORMS)
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_df_accuracy_guard(kernel, form):
    res = MATRIX_RUNNERS[kernel](2048, 2048, 2048, synth.KIND_UNIFORM, seed=7, form=form)
    _check(res, tol=1e-13)


@pytest.mark.parametrize("form", DF_FORMS)
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_df_integer_exact(kernel, form):
    scal = {"bicgk": {}, "atax": {"beta": 2.0}, "gemver": {"alpha": 2.0, "beta": -3.0},
            "gesummv": {"alpha": 2.0, "beta": -1.0}, "dgemv": {"alpha": 3.0, "beta": -2.0},
            "dgemvt": {"alpha": -1.0, "beta": 2.0}}[kernel]
    _check(MATRIX_RUNNERS[kernel](300, 517, 302, synth.KIND_INTEGER, seed=4, form=form, **scal), exact=True)


@pytest.mark.parametrize("form", ["df", "df_unfused"])
@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_df_unsuited_layout_runs_the_fp64_form(kernel, form):
    # Odd leading dimension: the tensor map cannot describe the matrix, so the
    # call runs the FP64 form, bit for bit.
    fp64 = "fused" if form == "df" else "unfused"
    a = MATRIX_RUNNERS[kernel](701, 333, 703, synth.KIND_UNIFORM, seed=3, form=form)
    b = MATRIX_RUNNERS[kernel](701, 333, 703, synth.KIND_UNIFORM, seed=3, form=fp64)
    for k in a:
        assert np.array_equal(a[k][0], b[k][0]), k


@pytest.mark.parametrize("kernel", sorted(MATRIX_RUNNERS))
def test_df_deterministic(kernel):
    a = MATRIX_RUNNERS[kernel](3001, 1778, 3002, synth.KIND_UNIFORM, seed=9, form="df")
    b = MATRIX_RUNNERS[kernel](3001, 1778, 3002, synth.KIND_UNIFORM, seed=9, form="df")
    for k in a:
        assert np.array_equal(a[k][0], b[k][0], equal_nan=True), k


def _compare_special(g, o, tol=TOL64):
    g, o = np.asarray(g, np.float64).ravel(), np.asarray(o, np.float64).ravel()
    assert np.array_equal(np.isnan(g), np.isnan(o)), "NaN positions differ"
    fin = np.isfinite(o)
    assert np.array_equal(g[~fin & ~np.isnan(o)], o[~fin & ~np.isnan(o)]), "Inf values differ"
    assert np.array_equal(np.isfinite(g), fin), "finite positions differ"
    if fin.any():
        scale = max(float(np.max(np.abs(o[fin]))), np.finfo(np.float64).tiny)   # keep the norms finite
        assert relerr(g[fin] / scale, o[fin] / scale) <= tol


def _special_matrix(m, n, lda, seed, plant):
    A = synth.matrix(seed, 0, m, n, lda=lda)
    for (i, j, v) in plant:
        A[i, j] = v
    return A


# Values planted at scattered positions (several chunks and panels); each
# case also has an exact zero.  "beyond" and "overflow" leave FP32's range.
PLANTS = {
    "zeros": [(i, j, 0.0) for i in range(0, 900, 7) for j in range(0, 600, 97)],
    "tiny": [(5, 3, 1e-30), (700, 400, -3e-25), (301, 599, 2.0 ** -71)],
    "large": [(17, 11, 1e25), (600, 123, -2.0 ** 61), (899, 0, 7e30)],
    "beyond": [(17, 11, 1e50), (600, 123, -2.0 ** 200), (899, 0, 3e300)],
    "overflow": [(300, 300, 3e37), (301, 300, 3e37), (302, 300, 3e37)],
    "nan": [(100, 50, np.nan)],
    "inf": [(256, 300, np.inf), (257, 301, -np.inf)],
    "denormal": [(44, 44, 5e-320), (45, 44, -1e-310)],
}


@pytest.mark.parametrize("case", sorted(PLANTS))
def test_df_range_fallback_bicgk_dgemv_gesummv_atax(case):
    m, n, lda = 900, 600, 900
    A = _special_matrix(m, n, lda, 21, PLANTS[case] + [(3, 3, 0.0)])
    pv, rv = synth.vector(21, 1, n), synth.vector(21, 2, m)
    dA = dev(A)
    q, s = Out(m), Out(n)
    w, nb = ws("bicgk", bto.BTO_FORM_DF, m, n)
    bto.bto_bicgk_df(m, n, p(dA), lda, dev(pv), dev(rv), q.ptr(), s.ptr(), p(w), nb, None)
    sync()
    assert bto.bto_device_status(p(w)) == 0
    qo, so = O.bicgk(m, n, A, pv, rv)
    _compare_special(q.host(), qo)
    _compare_special(s.host(), so)
    z = Out(m)
    w, nb = ws("dgemv", bto.BTO_FORM_DF, m, n)
    bto.bto_dgemv_df(m, n, 1.5, p(dA), lda, dev(pv), -0.5, dev(rv), z.ptr(), p(w), nb, None)
    sync()
    _compare_special(z.host(), O.dgemv(m, n, 1.5, A, pv, -0.5, rv))
    B2 = synth.matrix(21, 5, m, n, lda=lda)
    y = Out(m)
    w, nb = ws("gesummv", bto.BTO_FORM_DF, m, n)
    bto.bto_gesummv_df(m, n, 1.5, p(dev(B2)), lda, -0.75, p(dA), lda, dev(pv), y.ptr(), p(w), nb, None)
    sync()
    _compare_special(y.host(), O.gesummv(m, n, 1.5, B2, -0.75, A, pv))
    ya = Out(n)
    w, nb = ws("atax", bto.BTO_FORM_DF, m, n)
    bto.bto_atax_df(m, n, 1.25, p(dA), lda, dev(pv), ya.ptr(), p(w), nb, None)
    sync()
    _compare_special(ya.host(), O.atax(m, n, 1.25, A, pv))


@pytest.mark.parametrize("where", ["p", "r"])
@pytest.mark.parametrize("value", [1e-12, 3e12, 0.0, np.nan, 1e45, -np.inf, 1e-45])
def test_df_vector_range_fallback(where, value):
    m, n = 700, 500
    A = synth.matrix(22, 0, m, n)
    pv, rv = synth.vector(22, 1, n), synth.vector(22, 2, m)
    (pv if where == "p" else rv)[123] = value
    q, s = Out(m), Out(n)
    w, nb = ws("bicgk", bto.BTO_FORM_DF, m, n)
    bto.bto_bicgk_df(m, n, dev(A), m, dev(pv), dev(rv), q.ptr(), s.ptr(), p(w), nb, None)
    sync()
    qo, so = O.bicgk(m, n, A, pv, rv)
    _compare_special(q.host(), qo)
    _compare_special(s.host(), so)


@pytest.mark.parametrize("case", ["plain", "tiny", "huge", "nan", "vector"])
def test_df_gemver_in_place(case):
    # B written over A (and x over z), including lanes whose B elements take
    # the FP64 path because something they hold is out of range.
    m, n = 1100, 611
    ids = synth.GEMVER_IDS
    A = synth.matrix(2, ids["A"], m, n, lda=1100)
    plant = {"plain": [], "tiny": [(17, 5, 1e-40), (600, 300, 3e-29)], "huge": [(0, 0, 1e40), (1099, 610, -9e300)],
             "nan": [(513, 77, np.nan)], "vector": []}[case]
    for (i, j, v) in plant:
        A[i, j] = v
    vecs = [synth.vector(2, ids[k], m if k in ("u1", "u2", "y") else n) for k in ("u1", "v1", "u2", "v2", "y", "z")]
    if case == "vector":
        vecs[0][700] = 1e40       # u1 beyond FP32: those rows' B in FP64
        vecs[3][12] = np.inf      # v2 infinite: that column's B in FP64
    Bo, xo, wo = O.gemver(m, n, 1.5, 1.2, A, *vecs)
    dA = dev(A)
    d = [dev(v) for v in vecs]
    w = Out(m)
    wk, nb = ws("gemver", bto.BTO_FORM_DF, m, n)
    bto.bto_gemver_df(m, n, 1.5, 1.2, p(dA), 1100, *[p(t) for t in d], p(dA), 1100, p(d[5]), w.ptr(),
                      p(wk), nb, None)
    sync()
    assert bto.bto_device_status(p(wk)) == 0
    Bg = dA.cpu().numpy().reshape(n, 1100).T[:m]
    _compare_special(Bg, Bo, tol=1e-13)
    _compare_special(d[5].cpu().numpy(), xo)
    _compare_special(w.host(), wo)
    # B is formed by the FP64 form's two FMAs per element: the same bits as bto_gemver's.
    dA2 = dev(A)
    d2 = [dev(v) for v in vecs]
    B64 = torch.empty(1100 * n, dtype=torch.float64, device="cuda")
    x64, w64 = Out(n), Out(m)
    wk2, nb2 = ws("gemver", 0, m, n)
    bto.bto_gemver(m, n, 1.5, 1.2, p(dA2), 1100, *[p(t) for t in d2], p(B64), 1100, x64.ptr(), w64.ptr(),
                   p(wk2), nb2, None)
    sync()
    B64h = B64.cpu().numpy().reshape(n, 1100).T[:m]
    assert np.array_equal(Bg, B64h, equal_nan=True)


def test_df_zero_data_gives_exact_zeros():
    m, n = 514, 257
    Z = np.zeros((m, n))
    zv_n, zv_m = np.zeros(n), np.zeros(m)
    q, s = Out(m), Out(n)
    w, nb = ws("bicgk", bto.BTO_FORM_DF, m, n)
    bto.bto_bicgk_df(m, n, dev(Z), m, dev(synth.vector(1, 1, n)), dev(synth.vector(1, 2, m)), q.ptr(), s.ptr(),
                     p(w), nb, None)
    sync()
    assert np.all(q.host() == 0.0) and np.all(s.host() == 0.0)
    A = synth.matrix(1, 0, m, n)
    bto.bto_bicgk_df(m, n, dev(A), m, dev(zv_n), dev(zv_m), q.ptr(), s.ptr(), p(w), nb, None)
    sync()
    assert np.all(q.host() == 0.0) and np.all(s.host() == 0.0)


def test_df_workspace_and_form_queries():
    for k in sorted(MATRIX_RUNNERS):
        for form in (bto.BTO_FORM_DF, bto.BTO_FORM_DF_UNFUSED):
            nb = bto.bto_workspace_bytes(k, form, 4096, 3000)
            # Room for the FP64 form the call runs on unsuited layouts.
            fp = bto.bto_workspace_bytes(k, form - 2, 4096, 3000)
            assert nb >= fp > 0
    for k in ("axpydot", "waxpby", "vadd"):
        with pytest.raises(bto.BtoError) as e:
            bto.bto_workspace_bytes(k, bto.BTO_FORM_DF, 0, 1000)
        assert e.value.status == bto.BTO_ERR_UNSUPPORTED
    with pytest.raises(bto.BtoError) as e:
        bto.bto_workspace_bytes("bicgk", bto.BTO_FORM_DF, 100, 100, bto.BTO_F32)
    assert e.value.status == bto.BTO_ERR_UNSUPPORTED


def test_df_workspace_too_small_is_rejected():
    m, n = 100, 100
    A = dev(synth.matrix(1, 0, m, n))
    v = dev(synth.vector(1, 1, n))
    q, s = Out(m), Out(n)
    wk, nb = ws("bicgk", bto.BTO_FORM_DF, m, n)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_df(m, n, p(A), m, p(v), p(v), q.ptr(), s.ptr(), p(wk), nb - 8, None)
    assert e.value.status == bto.BTO_ERR_WORKSPACE and e.value.arg == 9


def test_df_ring_wait_expires_into_the_status_word():
    # Block 0's producer stops after one ring fill (its first tile has nine
    # stages here), so that block's consumer waits run out after 50 ms: the
    # status word reads BTO_ERR_TIMEOUT and the context stays usable.  The next
    # ordinary call clears the status and matches the oracle.  (An even
    # leading dimension, so that the double-float sweep takes the call.)
    m, n = 3000, 1778
    A = synth.matrix(23, 0, m, n)
    pv, rv = synth.vector(23, 1, n), synth.vector(23, 2, m)
    dA, dpv, drv = dev(A), dev(pv), dev(rv)
    q, s = Out(m), Out(n)
    w, nb = ws("bicgk", bto.BTO_FORM_DF, m, n)
    args = (m, n, p(dA), m, p(dpv), p(drv), q.ptr(), s.ptr(), p(w), nb)
    bto.bto_debug_df_stall(*args, 0, 50, None)
    sync()
    assert bto.bto_device_status(p(w)) == bto.BTO_ERR_TIMEOUT
    bto.bto_bicgk_df(*args, None)
    sync()
    assert bto.bto_device_status(p(w)) == 0
    qo, so = O.bicgk(m, n, A, pv, rv)
    assert relerr(q.host(), qo) < TOL64
    assert relerr(s.host(), so) < TOL64
