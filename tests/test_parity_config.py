"""Parity at the benchmarked sizes of the widened forms, in the launch
configuration the benchmark times:
- row-major storage at n = 16384 (bto_*_layout), sampled rows and columns;
- a generated program (the generator's BICGK and its two-matrix chain) at
  n = 16384, sampled;
- CSR BICGK and BATAX at 2^20 rows with 32 entries per row on average (the
  benchmark's sparse workload, 33.6 M entries), every output;
- the 4096-instance batched workload (m, n log-uniform in [32, 2048], FP32,
  leading dimensions padded to 16 bytes, 50/50 BICGK/GEMVER), 64 sampled
  instances checked on their stored values.
Matrices come from the device fill; the oracle recomputes sampled outputs
from the same generator's rows and columns on the host."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from gpu_util import TOL64, Out, dev, p, relerr, sync, ws
from paper_1205_1098_gb300 import _lib

pytestmark = pytest.mark.gpu

N = 16384
SEED = 1


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


def _samples(seed, n, k=32):
    return np.unique(np.concatenate([[0, n - 1, n // 2],
                                     (synth.vector(seed, 99, k) * 0.5 + 0.5) * (n - 1)]).astype(np.int64))


def test_row_major_bicgk_and_dgemv_n16384(A):
    # The buffer read as row-major is M = A^T: row i of M is column i of A.
    pv, rv = synth.vector(SEED, 1, N), synth.vector(SEED, 2, N)
    q, s = Out(N), Out(N)
    nb = bto.bto_layout_workspace_bytes("bicgk", _lib.BTO_ROW_MAJOR, 0, N, N)
    wk = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    bto.bto_bicgk_layout(_lib.BTO_ROW_MAJOR, N, N, p(A), N, dev(pv), dev(rv), q.ptr(), s.ptr(), p(wk), nb, None)
    sync()
    I, J = _samples(31, N), _samples(32, N)
    MI = synth.matrix_cols(SEED, 0, N, N, I).T          # rows I of M
    MJ = synth.matrix_rows(SEED, 0, N, N, J).T          # columns J of M
    qo = np.array([O.bicgk(1, N, MI[k:k + 1], pv, rv[i:i + 1])[0][0] for k, i in enumerate(I)])
    so = np.array([O.bicgk(N, 1, np.asfortranarray(MJ[:, k:k + 1]), pv[j:j + 1], rv)[1][0] for k, j in enumerate(J)])
    assert relerr(q.host()[I], qo) < TOL64 and relerr(s.host()[J], so) < TOL64
    # DGEMV with transposition on the same storage: z = alpha M^T x + beta y.
    z = Out(N)
    nb = bto.bto_layout_workspace_bytes("dgemv", _lib.BTO_ROW_MAJOR, _lib.BTO_TRANS, N, N)
    wk = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    bto.bto_dgemv_layout(_lib.BTO_ROW_MAJOR, _lib.BTO_TRANS, N, N, 1.5, p(A), N, dev(pv), -0.5, dev(rv), z.ptr(),
                         p(wk), nb, None)
    sync()
    zo = np.array([O.dgemv(1, N, 1.5, np.asfortranarray(MJ[:, k:k + 1].T), pv, -0.5, rv[j:j + 1])[0]
                   for k, j in enumerate(J)])
    assert relerr(z.host()[J], zo) < TOL64


@pytest.mark.parametrize("name", ["bicgk", "chain"])
def test_generated_program_n16384(A, name):
    from paper_1205_1098_gb300 import generator as G
    text = {"bicgk": "in: A : matrix, p r : vector\nout: q s : vector\nq = A * p\ns = A' * r",
            "chain": "in: A C : matrix, p r : vector\nout: q s v : vector\nq = A * p\ns = A' * r\nv = C * q + 2 * s"}[name]
    P = G.compile(text)
    f64 = dict(dtype=torch.float64, device="cuda")
    pv, rv = synth.vector(SEED, 1, N), synth.vector(SEED, 2, N)
    bind = {"A": A, "p": dev(pv), "r": dev(rv), "q": torch.empty(N, **f64), "s": torch.empty(N, **f64)}
    if name == "chain":
        bind["C"] = torch.empty(N * N, **f64)
        bto.bto_fill_f64(SEED, 5, 0, N, N, 0, p(bind["C"]), N, None)
        bind["v"] = torch.empty(N, **f64)
    prog, keep = P.program(bind, {k: (N, N) for k in ("A", "C") if k in bind})
    nb = bto.bto_program_workspace_bytes(prog)
    wk = torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda")
    bto.bto_program_run(prog, wk, nb, None)
    sync()
    I, J = _samples(33, N), _samples(34, N)
    RA, CA = synth.matrix_rows(SEED, 0, N, N, I), synth.matrix_cols(SEED, 0, N, N, J)
    q, s = bind["q"].cpu().numpy(), bind["s"].cpu().numpy()
    qo = np.array([O.bicgk(1, N, RA[k:k + 1], pv, rv[i:i + 1])[0][0] for k, i in enumerate(I)])
    so = np.array([O.bicgk(N, 1, CA[:, k:k + 1], pv[j:j + 1], rv)[1][0] for k, j in enumerate(J)])
    assert relerr(q[I], qo) < TOL64 and relerr(s[J], so) < TOL64
    if name == "chain":
        # v = C q + 2 s: rows I of C against the full q and s the program produced
        # (q and s themselves are checked above).
        RC = synth.matrix_rows(SEED, 5, N, N, I)
        vo = np.array([O.dgemv(1, N, 1.0, RC[k:k + 1], q, 2.0, s[i:i + 1])[0] for k, i in enumerate(I)])
        assert relerr(bind["v"].cpu().numpy()[I], vo) < TOL64
    del keep


def test_csr_2e20_rows():
    m, avg, seed = 1 << 20, 32, 11
    rp, col, val = synth.csr(seed, 70, m, m, avg)
    nnz = len(col)
    pv, rv = synth.vector(seed, 1, m), synth.vector(seed, 2, m)
    d_rp, d_col, d_val = (torch.from_numpy(a).cuda() for a in (rp, col, val))
    q, s, y = Out(m), Out(m), Out(m)
    nb = bto.bto_csr_workspace_bytes("atax", m, m, nnz)
    wk = torch.zeros(nb, dtype=torch.uint8, device="cuda")
    bto.bto_csr_bicgk(m, m, nnz, d_rp, d_col, d_val, dev(pv), dev(rv), q.ptr(), s.ptr(), wk, nb, None)
    bto.bto_csr_atax(m, m, nnz, d_rp, d_col, d_val, 0.75, dev(pv), y.ptr(), wk, nb, None)
    sync()
    assert int(wk[:4].view(torch.int32).cpu().numpy()[0]) == 0
    qo, so = O.csr_bicgk(m, m, rp, col, val, pv, rv)
    yo = O.csr_atax(m, m, 0.75, rp, col, val, pv)
    assert relerr(q.host(), qo) < TOL64 and relerr(s.host(), so) < TOL64 and relerr(y.host(), yo) < TOL64


def test_batched_config_4096_sampled():
    """The benchmark's batched workload, built the same way on the device."""
    count, seed = 4096, 3
    u = synth.vector(seed, 500, 2 * count) * 0.5 + 0.5
    sizes = np.round(np.exp(np.log(32) + u * (np.log(2048) - np.log(32)))).astype(np.int64)
    ops = np.where(synth.vector(seed, 501, count) < 0, 0, 2)
    descs = (bto.BatchDesc * count)()
    f32 = dict(dtype=torch.float32, device="cuda")
    keep, outs = [], []
    for i in range(count):
        m, n, op = int(sizes[2 * i]), int(sizes[2 * i + 1]), int(ops[i])
        d = descs[i]
        lda = (m + 3) // 4 * 4
        d.op, d.a_type, d.m, d.n, d.lda, d.ldb, d.alpha, d.beta = op, 1, m, n, lda, lda, 1.5, 1.25
        Ad = torch.empty(lda * n, **f32)
        bto.bto_fill_f32(seed, 1000 * i, 0, m, n, 0, Ad, lda, None)
        keep.append(Ad)
        d.A = Ad.data_ptr()
        for k, ln in enumerate([n, m] if op == 0 else [m, n, m, n, m, n]):
            t = torch.empty(ln, **f32)
            bto.bto_fill_f32(seed, 1000 * i + 1 + k, 0, ln, 1, 0, t, ln, None)
            keep.append(t)
            d.in_[k] = t.data_ptr()
        o = []
        for k, ln in enumerate([m, n] if op == 0 else [n, m]):
            t = torch.full((ln,), float("nan"), **f32)
            keep.append(t)
            d.out[k] = t.data_ptr()
            o.append(t)
        if op == 2:
            Bd = torch.empty(lda * n, **f32)
            keep.append(Bd)
            d.B = Bd.data_ptr()
            o.append(Bd)
        outs.append(o)
    nb = bto.bto_batch_workspace_bytes(descs, 512)
    wk = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    bto.bto_batch_prepare(count, descs, 512, wk, nb, None)
    bto.bto_batch_run(wk, nb, None)
    sync()
    assert bto.bto_device_status(wk) == 0
    f32h = lambda a64: synth.to_f32(a64).astype(np.float64)
    for i in np.unique(np.linspace(0, count - 1, 64).astype(np.int64)):
        m, n, op = int(sizes[2 * i]), int(sizes[2 * i + 1]), int(ops[i])
        lda = (m + 3) // 4 * 4
        Ah = f32h(synth.matrix(seed, 1000 * int(i), m, n))
        vin = [f32h(synth.vector(seed, 1000 * int(i) + 1 + k, ln))
               for k, ln in enumerate([n, m] if op == 0 else [m, n, m, n, m, n])]
        got = [t.cpu().numpy().astype(np.float64) for t in outs[i]]
        if op == 0:
            qo, so = O.bicgk(m, n, Ah, vin[0], vin[1])
            assert relerr(got[0], qo) <= 1e-6 and relerr(got[1], so) <= 1e-6, i
        else:
            # x and w from the B the call returned (formed in FP32 on the device).
            Bret = got[2][:lda * n].reshape(n, lda).T[:m]
            zm, zn = np.zeros(m), np.zeros(n)
            _, xo, wo = O.gemver(m, n, 1.5, 1.25, np.asfortranarray(Bret), zm, zn, zm, zn, vin[4], vin[5])
            Bex, _, _ = O.gemver(m, n, 1.5, 1.25, Ah, *vin)
            assert relerr(got[0], xo) <= 1e-6 and relerr(got[1], wo) <= 1e-6, i
            assert relerr(Bret, Bex) <= 1e-6, i
    del keep
