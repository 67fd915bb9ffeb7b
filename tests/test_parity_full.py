"""Parity at the benchmark's full sizes (n = 16384 matrices, 2^26 vectors),
in the launch configuration the benchmark times, for the FP64 form and the
double-float form of the matrix sequences.  Matrices are generated on
the device by the seeded fill; the oracle recomputes sampled outputs from
the same generator's rows and columns on the host, by running on the
sub-problem that determines each sampled output exactly."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from f64_cases import entry
from gpu_util import TOL64, Out, dev, p, relerr, sync, ws

pytestmark = pytest.mark.gpu

N = 16384
SEED = 1
NSAMP = 48
FORMS = ["fused", "df"]
# GEMVER's B: both forms compute A + u1 v1^T + u2 v2^T with two FP64 FMAs
# per element (the oracle rounds twice without contraction: a few ulps apart).
B_TOL = {"fused": 1e-15, "df": 1e-15}


@pytest.fixture(scope="module")
def A():
    from paper_1205_1098_gb300 import build
    build.build()
    t = torch.empty(N * N, dtype=torch.float64, device="cuda")
    bto.bto_fill_f64(SEED, 0, 0, N, N, 0, p(t), N, None)
    sync()
    yield t
    del t
    torch.cuda.empty_cache()


def _samples(seed, n, k=NSAMP):
    idx = np.unique(np.concatenate([[0, n - 1, n // 2],
                                    (synth.vector(seed, 99, k) * 0.5 + 0.5) * (n - 1)]).astype(np.int64))
    return idx


def _rows(aid, rows):
    return synth.matrix_rows(SEED, aid, N, N, rows)


def _cols(aid, cols):
    return synth.matrix_cols(SEED, aid, N, N, cols)


@pytest.mark.parametrize("form", FORMS)
def test_bicgk_full(A, form):
    pv, rv = synth.vector(SEED, 1, N), synth.vector(SEED, 2, N)
    q, s = Out(N), Out(N)
    wk, nb = ws("bicgk", entry("bicgk", form)[1], N, N)
    entry("bicgk", form)[0](N, N, p(A), N, dev(pv), dev(rv), q.ptr(), s.ptr(), p(wk), nb, None)
    sync()
    qh, sh = q.host(), s.host()
    I = _samples(11, N)
    R = _rows(0, I)
    qo = np.array([O.bicgk(1, N, R[k:k + 1], pv, rv[i:i + 1])[0][0] for k, i in enumerate(I)])
    C = _cols(0, I)
    so = np.array([O.bicgk(N, 1, C[:, k:k + 1], pv[j:j + 1], rv)[1][0] for k, j in enumerate(I)])
    assert relerr(qh[I], qo) < TOL64 and relerr(sh[I], so) < TOL64
    # adjoint identity over the whole outputs
    scale = np.linalg.norm(rv) * np.linalg.norm(pv) * N
    assert abs(np.dot(rv, qh) - np.dot(sh, pv)) < 1e-12 * scale


@pytest.mark.parametrize("form", FORMS)
def test_gesummv_full(A, form):
    Bm = torch.empty(N * N, dtype=torch.float64, device="cuda")
    bto.bto_fill_f64(SEED, 1, 0, N, N, 0, p(Bm), N, None)
    xv = synth.vector(SEED, 2, N)
    y = Out(N)
    wk, nb = ws("gesummv", entry("gesummv", form)[1], N, N)
    entry("gesummv", form)[0](N, N, 1.5, p(A), N, -0.75, p(Bm), N, dev(xv), y.ptr(), p(wk), nb, None)
    sync()
    del Bm
    I = _samples(12, N)
    RA, RB = _rows(0, I), _rows(1, I)
    yo = np.array([O.gesummv(1, N, 1.5, RA[k:k + 1], -0.75, RB[k:k + 1], xv)[0] for k in range(len(I))])
    assert relerr(y.host()[I], yo) < TOL64


@pytest.mark.parametrize("form", FORMS)
def test_dgemv_full(A, form):
    xv, yv = synth.vector(SEED, 1, N), synth.vector(SEED, 2, N)
    z = Out(N)
    wk, nb = ws("dgemv", entry("dgemv", form)[1], N, N)
    entry("dgemv", form)[0](N, N, 1.5, p(A), N, dev(xv), -0.5, dev(yv), z.ptr(), p(wk), nb, None)
    sync()
    I = _samples(13, N)
    R = _rows(0, I)
    zo = np.array([O.dgemv(1, N, 1.5, R[k:k + 1], xv, -0.5, yv[i:i + 1])[0] for k, i in enumerate(I)])
    assert relerr(z.host()[I], zo) < TOL64


def _gemver_vectors():
    ids = synth.GEMVER_IDS
    return {k: synth.vector(SEED, ids[k], N) for k in ("u1", "v1", "u2", "v2", "y", "z")}


@pytest.mark.parametrize("form", FORMS)
def test_gemver_full_dense(A, form):
    v = _gemver_vectors()
    B, x, w = Out(N * N), Out(N), Out(N)
    wk, nb = ws("gemver", entry("gemver", form)[1], N, N)
    entry("gemver", form)[0](N, N, 1.5, 1.2, p(A), N, *[dev(v[k]) for k in ("u1", "v1", "u2", "v2", "y", "z")],
                   B.ptr(), N, x.ptr(), w.ptr(), p(wk), nb, None)
    sync()
    J = _samples(14, N, 24)
    C = _cols(0, J)
    xh = x.host()
    Bt = B.t.view(N, N)      # Bt[j] is column j
    xs, xref = [], []
    for k, j in enumerate(J):
        Bo, xo, _ = O.gemver(N, 1, 1.5, 1.2, C[:, k:k + 1], v["u1"], v["v1"][j:j + 1], v["u2"],
                             v["v2"][j:j + 1], v["y"], v["z"][j:j + 1])
        assert relerr(Bt[j].cpu().numpy(), Bo[:, 0]) < B_TOL[form]
        xs.append(xh[j]); xref.append(xo[0])
    assert relerr(xs, xref) < TOL64
    del B


@pytest.mark.parametrize("form", FORMS)
def test_gemver_full_sparse_y(A, form):
    # With a single non-zero y_k, x = beta B_k,: y_k + z needs row k of B only,
    # and w_i = alpha B_i,: x needs row i: the oracle on the rows {k} U I is exact.
    v = _gemver_vectors()
    k0 = 12345
    yv = np.zeros(N)
    yv[k0] = v["y"][k0]
    B, x, w = Out(N * N), Out(N), Out(N)
    wk, nb = ws("gemver", entry("gemver", form)[1], N, N)
    entry("gemver", form)[0](N, N, 1.5, 1.2, p(A), N, dev(v["u1"]), dev(v["v1"]), dev(v["u2"]),
                   dev(v["v2"]), dev(yv), dev(v["z"]), B.ptr(), N, x.ptr(), w.ptr(),
                   p(wk), nb, None)
    sync()
    del B
    I = np.concatenate([[k0], _samples(15, N, 24)])
    R = _rows(0, I)
    sub = np.asfortranarray(R)
    Bo, xo, wo = O.gemver(len(I), N, 1.5, 1.2, sub, v["u1"][I], v["v1"], v["u2"][I], v["v2"],
                          yv[I], v["z"])
    assert relerr(x.host(), xo) < TOL64
    assert relerr(w.host()[I], wo) < TOL64


@pytest.mark.parametrize("form", FORMS)
def test_dgemvt_full(A, form):
    k0 = 777
    yv = np.zeros(N)
    yv[k0] = synth.vector(SEED, 1, N)[k0]
    zv = synth.vector(SEED, 2, N)
    x, w = Out(N), Out(N)
    wk, nb = ws("dgemvt", entry("dgemvt", form)[1], N, N)
    entry("dgemvt", form)[0](N, N, 1.5, 1.2, p(A), N, dev(yv), dev(zv), x.ptr(), w.ptr(), p(wk), nb, None)
    sync()
    I = np.concatenate([[k0], _samples(16, N, 24)])
    sub = np.asfortranarray(_rows(0, I))
    xo, wo = O.dgemvt(len(I), N, 1.5, 1.2, sub, yv[I], zv)
    assert relerr(x.host(), xo) < TOL64 and relerr(w.host()[I], wo) < TOL64
    # dense y: x_j needs column j only
    yd = synth.vector(SEED, 1, N)
    x2, w2 = Out(N), Out(N)
    entry("dgemvt", form)[0](N, N, 1.5, 1.2, p(A), N, dev(yd), dev(zv), x2.ptr(), w2.ptr(), p(wk), nb, None)
    sync()
    J = _samples(17, N, 24)
    C = _cols(0, J)
    xo2 = np.array([O.dgemvt(N, 1, 1.5, 1.2, C[:, k:k + 1], yd, zv[j:j + 1])[0][0] for k, j in enumerate(J)])
    assert relerr(x2.host()[J], xo2) < TOL64


@pytest.mark.parametrize("form", FORMS)
def test_atax_full(A, form):
    # Sparse x (4 non-zeros at K): t = A[:, K] x_K, y_j = beta A[:, j]^T t; the
    # oracle on the columns K U {j} gives y_j exactly.
    K = np.array([3, 4000, 9001, 16383])
    xv = np.zeros(N)
    xv[K] = synth.vector(SEED, 1, N)[K]
    y = Out(N)
    wk, nb = ws("atax", entry("atax", form)[1], N, N)
    entry("atax", form)[0](N, N, 1.5, p(A), N, dev(xv), y.ptr(), p(wk), nb, None)
    assert bto.bto_device_status(p(wk)) == 0
    yh = y.host()
    J = _samples(18, N, 32)
    CK = _cols(0, K)
    got, ref = [], []
    for j in J:
        cols = np.concatenate([CK, _cols(0, [j])], axis=1)
        xs = np.concatenate([xv[K], [xv[j] if j not in K else 0.0]])
        yo = O.atax(N, len(xs), 1.5, np.asfortranarray(cols), xs)
        got.append(yh[j]); ref.append(yo[-1] if j not in K else yo[list(K).index(j)])
    assert relerr(got, ref) < TOL64
    # dense x: the unfused form reads A twice; both forms must agree
    xd = synth.vector(SEED, 1, N)
    y1, y2 = Out(N), Out(N)
    entry("atax", form)[0](N, N, 1.0, p(A), N, dev(xd), y1.ptr(), p(wk), nb, None)
    uf = "unfused" if form == "fused" else "df_unfused"
    wk2, nb2 = ws("atax", entry("atax", uf)[1], N, N)
    entry("atax", uf)[0](N, N, 1.0, p(A), N, dev(xd), y2.ptr(), p(wk2), nb2, None)
    sync()
    assert relerr(y1.host(), y2.host()) < TOL64


@pytest.mark.parametrize("kernel", ["axpydot", "waxpby", "vadd"])
def test_vectors_full(kernel):
    from f64_cases import VECTOR_RUNNERS
    n = 1 << 26
    kw = {"compensated": True} if kernel == "axpydot" else {}
    res = VECTOR_RUNNERS[kernel](n, synth.KIND_UNIFORM, seed=SEED, **kw)
    for k, (g, o) in res.items():
        assert relerr(g, o) < TOL64, k
    torch.cuda.empty_cache()


def test_device_fill_matches_host_generator():
    from paper_1205_1098_gb300 import build
    build.build()
    m, n, ld = 37, 53, 41
    cs = synth.colscale(3, n)
    for kind in (synth.KIND_UNIFORM, synth.KIND_INTEGER):
        for scale in (None, cs):
            ref = synth.matrix(3, 5, m, n, lda=ld, kind=kind, scale=scale)
            dcs = dev(scale) if scale is not None else None
            t = torch.full((ld * n,), np.nan, dtype=torch.float64, device="cuda")
            bto.bto_fill_f64(3, 5, kind, m, n, p(dcs), p(t), ld, None)
            f = torch.zeros(ld * n, dtype=torch.float32, device="cuda")
            bto.bto_fill_f32(3, 5, kind, m, n, p(dcs), p(f), ld, None)
            b = torch.zeros(ld * n, dtype=torch.int16, device="cuda")
            bto.bto_fill_bf16(3, 5, kind, m, n, p(dcs), p(b), ld, None)
            sync()
            got = t.cpu().numpy().reshape(n, ld).T[:m]
            assert np.array_equal(got, ref[:m])
            assert np.array_equal(f.cpu().numpy().reshape(n, ld).T[:m], synth.to_f32(ref[:m]))
            assert np.array_equal(b.cpu().numpy().view(np.uint16).reshape(n, ld).T[:m],
                                  synth.to_bf16_bits(ref[:m]))
