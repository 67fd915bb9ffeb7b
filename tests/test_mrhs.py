"""GPU parity of the multi-right-hand-side BICGK on the tensor cores
(Q = A P, S = A^T R; A, P, R BF16; Q, S FP32) against the FP64 oracle run on
the stored BF16 values.

Bounds: the tensor cores form BF16 x BF16 products exactly in FP32 and
accumulate in FP32 over each 512-column panel (Q) or each block's row range
(S); the per-panel and per-block partials are then added in compensated FP32
(TwoSum).  The FP32 rounding error of an n-term sum is at most (n-1) u32
times its absolute sum (u32 = 2^-24), and with signed uniform inputs the
rounding errors behave like a random walk, so the normwise error per
right-hand side stays well below 1e-5 (the test's tolerance) at every size
used here.  Integer-valued inputs with |values| <= 8 keep every partial sum
below 2^24 and are exact."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from gpu_util import GUARD, CANARY, p, sync

pytestmark = pytest.mark.gpu

TOL_MRHS = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


def bf16(a64):
    """FP64 array -> (BF16 bits as uint16, FP64 value of the stored BF16)."""
    nan = np.isnan(a64)
    bits = synth.to_bf16_bits(np.where(nan, 0.0, a64))
    bits = np.where(nan, np.uint16(0x7FC0), bits).astype(np.uint16)
    return bits, synth.bf16_bits_to_f64(bits)


def to_dev(bits):
    flat = np.ascontiguousarray(bits.ravel(order="F"))
    return torch.from_numpy(flat.view(np.int16)).cuda()


class Mat32:
    """Device FP32 output of rows x k (leading dimension ld) between canaries."""

    def __init__(self, rows, k, ld):
        self.rows, self.k, self.ld = rows, k, ld
        n = ld * k
        self.buf = torch.full((n + 2 * GUARD,), CANARY, dtype=torch.float32, device="cuda")
        self.t = self.buf[GUARD:GUARD + n]
        self.t.fill_(float("nan"))

    def ptr(self):
        return self.t.data_ptr() if self.rows * self.k else 0

    def host(self):
        g = self.buf.cpu().numpy()
        assert np.all(g[:GUARD] == CANARY) and np.all(g[GUARD + self.ld * self.k:] == CANARY), "guard overwritten"
        return g[GUARD:GUARD + self.ld * self.k].reshape(self.k, self.ld).T[:self.rows].astype(np.float64)


def workspace(m, n, k):
    nb = bto.bto_bicgk_mrhs_workspace_bytes(m, n, k)
    t = torch.empty(max(nb, 1) + 256, dtype=torch.uint8, device="cuda")
    t.fill_(0xA5)   # arbitrary content: the kernels must not depend on it
    return t, nb


def colerr(got, ref):
    """Largest normwise relative error over the right-hand sides (columns)."""
    if ref.size == 0:
        return 0.0
    e = 0.0
    for j in range(ref.shape[1]):
        nr = np.linalg.norm(ref[:, j])
        d = np.linalg.norm(got[:, j] - ref[:, j])
        e = max(e, d / nr if nr > 0 else d)
    return e


def run(m, n, k, lda=None, ldq=None, lds=None, kind=synth.KIND_UNIFORM, seed=3, pad_nan=True):
    lda = lda or max(1, m)
    A64 = synth.matrix(seed, 0, m, n, lda=lda, kind=kind, pad=np.nan if pad_nan else 0.0)
    Ab, Aq = bf16(A64)
    Pb, Pq = bf16(synth.matrix(seed, 1, n, k, kind=kind)) if n else (np.zeros((0, k), np.uint16), np.zeros((0, k)))
    Rb, Rq = bf16(synth.matrix(seed, 2, m, k, kind=kind)) if m else (np.zeros((0, k), np.uint16), np.zeros((0, k)))
    dA = to_dev(Ab) if m * n else None
    dP = to_dev(Pb) if n else None
    dR = to_dev(Rb) if m else None
    ldq, lds = ldq or max(1, m), lds or max(1, n)
    Q, S = Mat32(m, k, ldq), Mat32(n, k, lds)
    wk, nb = workspace(m, n, k)
    bto.bto_bicgk_mrhs(m, n, k, p(dA), lda, p(dP), max(1, n), p(dR), max(1, m), Q.ptr(), ldq, S.ptr(), lds,
                       p(wk), nb, None)
    sync()
    Qo, So = O.bicgk_mrhs(m, n, k, Aq[:m] if m else np.zeros((1, n)), Pq, Rq)
    return Q.host(), Qo, S.host(), So


# Shapes whose leading dimensions are multiples of 8 take the TMA kernel, the
# others the cp.async kernel; both sets cover ragged row tiles and panels.
SHAPES = [(1, 1, 16), (37, 129, 16), (300, 517, 48), (513, 1537, 64), (1000, 3001, 64), (4099, 250, 96),
          (129, 1031, 96),
          (8, 8, 32), (128, 512, 32), (520, 1544, 16), (1000, 3000, 64), (2048, 2048, 80), (4096, 248, 96),
          (136, 2056, 48)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_mrhs(shape):
    m, n, k = shape
    Q, Qo, S, So = run(m, n, k)
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(S))
    assert colerr(Q, Qo) <= TOL_MRHS and colerr(S, So) <= TOL_MRHS


def test_mrhs_integer_exact():
    for (m, n, k) in [(300, 517, 32), (1000, 1100, 64), (4099, 250, 16), (1000, 1104, 64), (2056, 520, 96)]:
        Q, Qo, S, So = run(m, n, k, kind=synth.KIND_INTEGER)
        assert np.array_equal(Q, Qo) and np.array_equal(S, So)


def test_mrhs_leading_dimensions_and_slow_path():
    # lda not a multiple of 8 takes the cp.async kernel (and its element-wise
    # copies for A); lda = 48 with aligned P, R takes the TMA kernel.  Both
    # issue the same MMAs in the same order: the same bits.
    m, n, k = 40, 704, 32
    Q, Qo, S, So = run(m, n, k, lda=45, ldq=41, lds=707)
    assert colerr(Q, Qo) <= TOL_MRHS and colerr(S, So) <= TOL_MRHS
    Q2, _, S2, _ = run(m, n, k, lda=48, ldq=41, lds=707)
    assert np.array_equal(Q, Q2) and np.array_equal(S, S2)
    Q3, _, S3, _ = run(1000, 3000, 64, lda=1003)
    Q4, _, S4, _ = run(1000, 3000, 64, lda=1000)
    assert np.array_equal(Q3, Q4) and np.array_equal(S3, S4)


def test_mrhs_output_gaps_untouched():
    m, n, k = 100, 300, 16
    lda, ldq, lds = 104, 103, 305
    A64 = synth.matrix(4, 0, m, n, lda=lda)
    Ab, _ = bf16(A64)
    Pb, _ = bf16(synth.matrix(4, 1, n, k))
    Rb, _ = bf16(synth.matrix(4, 2, m, k))
    Q, S = Mat32(m, k, ldq), Mat32(n, k, lds)
    wk, nb = workspace(m, n, k)
    bto.bto_bicgk_mrhs(m, n, k, to_dev(Ab), lda, to_dev(Pb), n, to_dev(Rb), m, Q.ptr(), ldq, S.ptr(), lds,
                       p(wk), nb, None)
    sync()
    gq = Q.t.cpu().numpy().reshape(k, ldq)
    gs = S.t.cpu().numpy().reshape(k, lds)
    assert np.all(np.isnan(gq[:, m:])) and np.all(np.isfinite(gq[:, :m]))
    assert np.all(np.isnan(gs[:, n:])) and np.all(np.isfinite(gs[:, :n]))


@pytest.mark.parametrize("shape", [(1000, 3001, 64), (1000, 3000, 64)], ids=["ldg", "tma"])
def test_mrhs_deterministic(shape):
    a = run(*shape, seed=9)
    b = run(*shape, seed=9)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("shape", [(0, 700, 16), (700, 0, 32), (0, 0, 16)])
def test_mrhs_empty(shape):
    m, n, k = shape
    Q, Qo, S, So = run(m, n, k)
    assert np.array_equal(Q, np.zeros((m, k))) and np.array_equal(S, np.zeros((n, k)))


def test_mrhs_rejects_bad_arguments():
    dummy = torch.zeros(1024, dtype=torch.int16, device="cuda")
    for k in (0, 8, 17, 112):
        with pytest.raises(bto.BtoError) as e:
            bto.bto_bicgk_mrhs(16, 16, k, p(dummy), 16, p(dummy), 16, p(dummy), 16, p(dummy), 16, p(dummy), 16,
                               0, 0, None)
        assert e.value.arg == 3
    wk, nb = workspace(64, 64, 16)
    Q, S = Mat32(64, 16, 64), Mat32(64, 16, 64)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_mrhs(64, 64, 16, p(dummy), 64, p(dummy), 64, p(dummy), 64, Q.ptr(), 64, S.ptr(), 64,
                           p(wk), nb - 256, None)
    assert e.value.status == bto.BTO_ERR_WORKSPACE and e.value.arg == 14


# ------------------------------------------------ 8192 x 8192, k = 64 (sampled)
NF, KF = 8192, 64


def test_mrhs_full_sampled():
    A = torch.empty(NF * NF, dtype=torch.int16, device="cuda")
    bto.bto_fill_bf16(6, 0, 0, NF, NF, 0, p(A), NF, None)
    Pb, Pq = bf16(synth.matrix(6, 1, NF, KF))
    Rb, Rq = bf16(synth.matrix(6, 2, NF, KF))
    Q, S = Mat32(NF, KF, NF), Mat32(NF, KF, NF)
    wk, nb = workspace(NF, NF, KF)
    bto.bto_bicgk_mrhs(NF, NF, KF, p(A), NF, to_dev(Pb), NF, to_dev(Rb), NF, Q.ptr(), NF, S.ptr(), NF,
                       p(wk), nb, None)
    sync()
    st = bto.bto_device_status(wk)
    del A
    torch.cuda.empty_cache()
    assert st == 0
    Qh, Sh = Q.host(), S.host()
    I = np.linspace(0, NF - 1, 24).astype(np.int64)
    rows = bf16(synth.matrix_rows(6, 0, NF, NF, I))[1]
    cols = bf16(synth.matrix_cols(6, 0, NF, NF, I))[1]
    for t, i in enumerate(I):
        qo = O.bicgk_mrhs(1, NF, KF, rows[t:t + 1], Pq, Rq[i:i + 1])[0][0]
        so = O.bicgk_mrhs(NF, 1, KF, cols[:, t:t + 1], Pq[i:i + 1], Rq)[1][0]
        assert np.linalg.norm(Qh[i] - qo) <= TOL_MRHS * np.linalg.norm(qo)
        assert np.linalg.norm(Sh[i] - so) <= TOL_MRHS * np.linalg.norm(so)
