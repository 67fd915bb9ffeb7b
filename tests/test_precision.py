"""GPU parity of the reduced-precision storage form (A in FP32 or BF16,
FP32 vectors, compensated FP32 accumulation, FP64 final combine) against the
FP64 oracle run on the stored values.  Bound: normwise relative error
<= 1e-6 per output; integer-valued inputs are exact; GEMVER's stored B is
within one storage-type ulp plus the FP32 evaluation error of the FP64 B,
and x, w are checked against the oracle run on the returned B."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from gpu_util import Out, dev, p, relerr, sync, ws

pytestmark = pytest.mark.gpu

TOL_LP = 1e-6
TYPES = {"f32": bto.BTO_F32, "bf16": bto.BTO_BF16}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


def quantize(a64, t):
    """FP64 array -> (stored numpy array in the storage type, its FP64 value)."""
    if t == "f32":
        q = synth.to_f32(a64)
        return q, q.astype(np.float64)
    nan = np.isnan(a64)
    bits = synth.to_bf16_bits(np.where(nan, 0.0, a64))
    bits = np.where(nan, np.uint16(0x7FC0), bits).astype(np.uint16)   # keep NaN padding as BF16 NaN
    return bits, synth.bf16_bits_to_f64(bits)


def dev_stored(q, t):
    flat = np.ascontiguousarray(q.ravel(order="F") if q.ndim == 2 else q)
    if t == "f32":
        return torch.from_numpy(flat).cuda()
    return torch.from_numpy(flat.view(np.int16)).cuda()


def host_stored(tensor, t):
    a = tensor.cpu().numpy()
    return a.astype(np.float64) if t == "f32" else synth.bf16_bits_to_f64(a.view(np.uint16))


def f32vec(seed, aid, n, kind=synth.KIND_UNIFORM):
    return synth.to_f32(synth.vector(seed, aid, n, kind))


def out32(n):
    return Out(n, dtype=torch.float32)


SHAPES = [(1, 1, 1), (3, 5, 3), (37, 129, 40), (300, 517, 300), (2048, 2048, 2048),
          (1000, 3001, 1003), (4099, 250, 4104), (0, 7, 1), (7, 0, 7)]


def run_bicgk_ex(t, m, n, lda, kind=synth.KIND_UNIFORM, seed=2, scale=None):
    A64 = synth.matrix(seed, 0, m, n, lda=lda, kind=kind, scale=scale)
    Aq, Adq = quantize(A64, t)
    pv, rv = f32vec(seed, 1, n, kind), f32vec(seed, 2, m, kind)
    dA, dp, dr = dev_stored(Aq, t), dev(pv, torch.float32), dev(rv, torch.float32)
    q, s = out32(m), out32(n)
    wk, nb = ws("bicgk", 0, m, n, TYPES[t])
    bto.bto_bicgk_ex(m, n, TYPES[t], p(dA), lda, p(dp), p(dr), q.ptr(), s.ptr(), p(wk), nb, None)
    sync()
    qo, so = O.bicgk(m, n, Adq[:m] if m else np.zeros((1, n)), pv.astype(np.float64), rv.astype(np.float64))
    return {"q": (q.host(), qo), "s": (s.host(), so)}


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("t", sorted(TYPES))
def test_bicgk_ex(t, shape):
    for k, (g, o) in run_bicgk_ex(t, *shape).items():
        assert relerr(g, o) <= TOL_LP, (k, relerr(g, o))


@pytest.mark.parametrize("t", sorted(TYPES))
def test_bicgk_ex_integer_exact(t):
    for k, (g, o) in run_bicgk_ex(t, 300, 517, 304, kind=synth.KIND_INTEGER).items():
        assert np.array_equal(g.astype(np.float64), o), k


@pytest.mark.parametrize("t", sorted(TYPES))
def test_bicgk_ex_column_scaled(t):
    m, n = 1500, 1200
    cs = synth.colscale(3, n)
    for k, (g, o) in run_bicgk_ex(t, m, n, m, scale=cs, seed=3).items():
        assert relerr(g, o) <= TOL_LP, (k, relerr(g, o))


def run_gemver_ex(t, m, n, lda, kind=synth.KIND_UNIFORM, seed=2, alpha=1.5, beta=1.2, scale=None):
    ids = synth.GEMVER_IDS
    A64 = synth.matrix(seed, ids["A"], m, n, lda=lda, kind=kind, scale=scale)
    Aq, _ = quantize(A64, t)
    vec = {k: f32vec(seed, ids[k], m if k in ("u1", "u2", "y") else n, kind)
           for k in ("u1", "v1", "u2", "v2", "y", "z")}
    dA = dev_stored(Aq, t)
    dv = [dev(vec[k], torch.float32) for k in ("u1", "v1", "u2", "v2", "y", "z")]
    Bt = torch.zeros(max(lda * n, 1), dtype=torch.float32 if t == "f32" else torch.int16, device="cuda")
    x, w = out32(n), out32(m)
    wk, nb = ws("gemver", 0, m, n, TYPES[t])
    bto.bto_gemver_ex(m, n, alpha, beta, TYPES[t], p(dA), lda, *[p(d) for d in dv], p(Bt), lda,
                      x.ptr(), w.ptr(), p(wk), nb, None)
    sync()
    Bret = host_stored(Bt, t)[:lda * n].reshape((n, lda)).T[:m] if n else np.zeros((m, 0))
    v64 = {k: v.astype(np.float64) for k, v in vec.items()}
    Adq = quantize(A64, t)[1]
    Bexact, _, _ = O.gemver(m, n, alpha, beta, Adq[:m] if m else np.zeros((1, n)), v64["u1"], v64["v1"],
                            v64["u2"], v64["v2"], v64["y"], v64["z"])
    zm, zn = np.zeros(m), np.zeros(n)
    _, xo, wo = O.gemver(m, n, alpha, beta, Bret if m else np.zeros((1, n)), zm, zn, zm, zn,
                         v64["y"], v64["z"])
    mag = (np.abs(Adq[:m]) + np.abs(np.outer(v64["u1"], v64["v1"])) + np.abs(np.outer(v64["u2"], v64["v2"])))
    return Bret, Bexact, mag, {"x": (x.host(), xo), "w": (w.host(), wo)}


def _b_ok(Bret, Bexact, mag, t):
    """B is formed in FP32 with two roundings (two fused multiply-adds), then
    rounded to the storage type: |B - B_exact| <= one storage ulp of B_exact
    plus the FP32 evaluation error 2 * 2^-24 * (|a| + |u1 v1| + |u2 v2|)."""
    ulp = np.spacing(np.abs(Bexact).astype(np.float32)).astype(np.float64)
    if t == "bf16":
        ulp = ulp * 2.0 ** 16
    return np.all(np.abs(Bret - Bexact) <= ulp + 2.0 ** -23 * mag)


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("t", sorted(TYPES))
def test_gemver_ex(t, shape):
    m, n, lda = shape
    Bret, Bexact, mag, res = run_gemver_ex(t, m, n, lda)
    assert _b_ok(Bret, Bexact, mag, t)
    for k, (g, o) in res.items():
        assert relerr(g, o) <= TOL_LP, (k, relerr(g, o))


@pytest.mark.parametrize("t", sorted(TYPES))
def test_gemver_ex_integer_b_and_x_exact(t):
    Bret, Bexact, _, res = run_gemver_ex(t, 300, 517, 304, kind=synth.KIND_INTEGER, alpha=2.0, beta=-3.0)
    assert np.array_equal(Bret, Bexact)
    assert np.array_equal(res["x"][0].astype(np.float64), res["x"][1])
    assert relerr(*res["w"]) <= TOL_LP


@pytest.mark.parametrize("t", sorted(TYPES))
def test_gemver_ex_column_scaled(t):
    cs = synth.colscale(4, 900)
    Bret, Bexact, mag, res = run_gemver_ex(t, 1100, 900, 1100, seed=4, scale=cs)
    assert _b_ok(Bret, Bexact, mag, t)
    for k, (g, o) in res.items():
        assert relerr(g, o) <= TOL_LP, (k, relerr(g, o))


def run_atax_ex(t, m, n, lda, kind=synth.KIND_UNIFORM, seed=2, beta=1.25, scale=None):
    A64 = synth.matrix(seed, 0, m, n, lda=lda, kind=kind, scale=scale)
    Aq, Adq = quantize(A64, t)
    xv = f32vec(seed, 1, n, kind)
    dA, dx = dev_stored(Aq, t), dev(xv, torch.float32)
    y = out32(n)
    wk, nb = ws("atax", 0, m, n, TYPES[t])
    bto.bto_atax_ex(m, n, beta, TYPES[t], p(dA), lda, p(dx), y.ptr(), p(wk), nb, None)
    sync()
    yo = O.atax(m, n, beta, Adq[:m] if m else np.zeros((1, n)), xv.astype(np.float64))
    return y.host(), yo


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("t", sorted(TYPES))
def test_atax_ex(t, shape):
    g, o = run_atax_ex(t, *shape)
    assert relerr(g, o) <= TOL_LP, relerr(g, o)


@pytest.mark.parametrize("t", sorted(TYPES))
def test_atax_ex_integer_exact(t):
    # n = 100 keeps every FP32 partial of the second sweep below 2^24.
    g, o = run_atax_ex(t, 300, 100, 304, kind=synth.KIND_INTEGER, beta=-2.0)
    assert np.array_equal(g.astype(np.float64), o)


@pytest.mark.parametrize("t", sorted(TYPES))
def test_atax_ex_column_scaled(t):
    cs = synth.colscale(6, 1300)
    g, o = run_atax_ex(t, 1700, 1300, 1700, seed=6, scale=cs)
    assert relerr(g, o) <= TOL_LP, relerr(g, o)


def run_gesummv_ex(t, m, n, lda, kind=synth.KIND_UNIFORM, seed=2, alpha=1.5, beta=-0.75, scale=None):
    A64 = synth.matrix(seed, 0, m, n, lda=lda, kind=kind, scale=scale)
    B64 = synth.matrix(seed, 1, m, n, lda=lda, kind=kind, scale=scale)
    (Aq, Adq), (Bq, Bdq) = quantize(A64, t), quantize(B64, t)
    xv = f32vec(seed, 2, n, kind)
    dA, dB, dx = dev_stored(Aq, t), dev_stored(Bq, t), dev(xv, torch.float32)
    y = out32(m)
    wk, nb = ws("gesummv", 0, m, n, TYPES[t])
    bto.bto_gesummv_ex(m, n, alpha, beta, TYPES[t], p(dA), lda, p(dB), lda, p(dx), y.ptr(), p(wk), nb, None)
    sync()
    z = np.zeros((1, n))
    yo = O.gesummv(m, n, alpha, Adq[:m] if m else z, beta, Bdq[:m] if m else z, xv.astype(np.float64))
    return y.host(), yo


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
@pytest.mark.parametrize("t", sorted(TYPES))
def test_gesummv_ex(t, shape):
    g, o = run_gesummv_ex(t, *shape)
    assert relerr(g, o) <= TOL_LP, relerr(g, o)


@pytest.mark.parametrize("t", sorted(TYPES))
def test_gesummv_ex_integer_exact(t):
    g, o = run_gesummv_ex(t, 300, 517, 304, kind=synth.KIND_INTEGER, alpha=2.0, beta=-3.0)
    assert np.array_equal(g.astype(np.float64), o)


@pytest.mark.parametrize("t", sorted(TYPES))
def test_gesummv_ex_column_scaled(t):
    cs = synth.colscale(7, 1100)
    g, o = run_gesummv_ex(t, 900, 1100, 904, seed=7, scale=cs)
    assert relerr(g, o) <= TOL_LP, relerr(g, o)


# ------------------------------------------------------------ n = 32768 (sampled)
NF = 32768


def _fill(t, scale_dev):
    fn = bto.bto_fill_f32 if t == "f32" else bto.bto_fill_bf16
    A = torch.empty(NF * NF, dtype=torch.float32 if t == "f32" else torch.int16, device="cuda")
    fn(5, 0, 0, NF, NF, p(scale_dev) if scale_dev is not None else 0, p(A), NF, None)
    return A


@pytest.mark.parametrize("scaled", [False, True], ids=["plain", "colscaled"])
@pytest.mark.parametrize("t", sorted(TYPES))
def test_bicgk_ex_full(t, scaled):
    cs = synth.colscale(5, NF) if scaled else None
    dcs = dev(cs) if scaled else None
    A = _fill(t, dcs)
    pv, rv = f32vec(5, 1, NF), f32vec(5, 2, NF)
    q, s = out32(NF), out32(NF)
    wk, nb = ws("bicgk", 0, NF, NF, TYPES[t])
    bto.bto_bicgk_ex(NF, NF, TYPES[t], p(A), NF, dev(pv, torch.float32), dev(rv, torch.float32),
                     q.ptr(), s.ptr(), p(wk), nb, None)
    sync()
    del A
    torch.cuda.empty_cache()
    I = np.linspace(0, NF - 1, 40).astype(np.int64)
    R = quantize(synth.matrix_rows(5, 0, NF, NF, I, scale=cs), t)[1]
    C = quantize(synth.matrix_cols(5, 0, NF, NF, I, scale=cs), t)[1]
    p64, r64 = pv.astype(np.float64), rv.astype(np.float64)
    qo = np.array([O.bicgk(1, NF, R[k:k + 1], p64, r64[i:i + 1])[0][0] for k, i in enumerate(I)])
    so = np.array([O.bicgk(NF, 1, C[:, k:k + 1], p64[j:j + 1], r64)[1][0] for k, j in enumerate(I)])
    assert relerr(q.host()[I], qo) <= TOL_LP and relerr(s.host()[I], so) <= TOL_LP


@pytest.mark.parametrize("t", sorted(TYPES))
def test_gemver_ex_full_sparse_y(t):
    ids = synth.GEMVER_IDS
    A = _fill(t, None)
    vec = {k: f32vec(5, ids[k], NF) for k in ("u1", "v1", "u2", "v2", "z")}
    k0 = 23456
    yv = np.zeros(NF, dtype=np.float32)
    yv[k0] = f32vec(5, ids["y"], NF)[k0]
    dv = [dev(vec[k], torch.float32) for k in ("u1", "v1", "u2", "v2")] + \
         [dev(yv, torch.float32), dev(vec["z"], torch.float32)]
    B = torch.empty(NF * NF, dtype=A.dtype, device="cuda")
    x, w = out32(NF), out32(NF)
    wk, nb = ws("gemver", 0, NF, NF, TYPES[t])
    bto.bto_gemver_ex(NF, NF, 1.5, 1.2, TYPES[t], p(A), NF, *[p(d) for d in dv], p(B), NF,
                      x.ptr(), w.ptr(), p(wk), nb, None)
    sync()
    del A
    I = np.concatenate([[k0], np.linspace(0, NF - 1, 20).astype(np.int64)])
    rows = B.view(NF, NF)[:, torch.from_numpy(I).cuda()].T.contiguous()     # rows I of B
    Brows = host_stored(rows, t).reshape(len(I), NF)
    del B
    torch.cuda.empty_cache()
    z64 = vec["z"].astype(np.float64)
    zm = np.zeros(len(I))
    _, xo, wo = O.gemver(len(I), NF, 1.5, 1.2, np.asfortranarray(Brows), zm, np.zeros(NF), zm,
                         np.zeros(NF), yv[I].astype(np.float64), z64)
    assert relerr(x.host(), xo) <= TOL_LP
    assert relerr(w.host()[I], wo) <= TOL_LP
