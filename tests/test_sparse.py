"""Sparse (CSR) BICGK and BATAX: the oracle's CSR definitions are pinned to
the dense oracle on the densified matrix, to a hand-worked example and to
closed forms; the C entry points validate their arguments without a GPU;
on the GPU both match the oracle, the row products are bitwise
reproducible, and malformed index data is skipped and reported through the
status word instead of being dereferenced."""
import numpy as np
import pytest

import golden_io
import oracle as O
import synth
import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import _lib, build


def _dense(m, n, rp, col, val):
    A = np.zeros((max(m, 1), n))
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            A[i, col[k]] += val[k]
    return np.asfortranarray(A[:m])


# ------------------------------------------------------------------ oracle pins


def test_csr_oracle_matches_dense_oracle():
    for (m, n, avg, seed) in ((30, 20, 4, 1), (7, 50, 12, 2), (40, 3, 2, 3), (5, 5, 0, 4)):
        rp, col, val = synth.csr(seed, 60, m, n, avg)
        A = _dense(m, n, rp, col, val)
        p, r = synth.vector(seed, 1, n), synth.vector(seed, 2, m)
        q, s = O.csr_bicgk(m, n, rp, col, val, p, r)
        qd, sd = O.bicgk(m, n, A, p, r)
        assert np.allclose(q, qd, rtol=0, atol=1e-13) and np.allclose(s, sd, rtol=0, atol=1e-13)
        y = O.csr_atax(m, n, 1.5, rp, col, val, p)
        assert np.allclose(y, O.atax(m, n, 1.5, A, p), rtol=0, atol=1e-12)


def test_csr_oracle_hand_worked():
    inp, exp = golden_io.load("csr_bicgk_3x4.txt")
    m, n = inp["m"], inp["n"]
    rp, col = inp["row_ptr"].astype(np.int64), inp["col"].astype(np.int32)
    q, s = O.csr_bicgk(m, n, rp, col, inp["val"], inp["p"], inp["r"])
    assert np.array_equal(q, exp["q"]) and np.array_equal(s, exp["s"])
    y = O.csr_atax(m, n, float(inp["beta"]), rp, col, inp["val"], inp["p"])
    assert np.array_equal(y, exp["y"])


def test_csr_oracle_closed_forms():
    n = 9
    rp, col, val = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n)
    p, r = np.arange(1.0, n + 1), np.arange(-4.0, n - 4)
    q, s = O.csr_bicgk(n, n, rp, col, val, p, r)
    assert np.array_equal(q, p) and np.array_equal(s, r)            # identity
    assert np.array_equal(O.csr_atax(n, n, 3.0, rp, col, val, p), 3.0 * p)
    # Duplicated entries add: row 0 holds (0, 0) twice with values 1 and 2.
    q, s = O.csr_bicgk(1, 1, np.array([0, 2]), np.array([0, 0], np.int32), np.array([1.0, 2.0]),
                       np.array([5.0]), np.array([7.0]))
    assert q[0] == 15.0 and s[0] == 21.0


# ------------------------------------------------------------------ CPU validation


def test_csr_validation_without_gpu():
    build.build()
    with pytest.raises(bto.BtoError) as e:
        bto.bto_csr_bicgk(-1, 4, 0, 4096, 8192, 12288, 16384, 20480, 24576, 28672, 0, 256, 0)
    assert e.value.arg == 1
    with pytest.raises(bto.BtoError) as e:     # n beyond int32 column indices
        bto.bto_csr_bicgk(4, 1 << 31, 0, 4096, 8192, 12288, 16384, 20480, 24576, 28672, 0, 256, 0)
    assert e.value.arg == 2
    with pytest.raises(bto.BtoError) as e:     # NULL row pointers with rows
        bto.bto_csr_bicgk(4, 4, 3, 0, 8192, 12288, 16384, 20480, 24576, 28672, 0, 256, 0)
    assert e.value.arg == 4
    with pytest.raises(bto.BtoError) as e:     # q overlapping s
        bto.bto_csr_bicgk(4, 4, 3, 4096, 8192, 12288, 16384, 20480, 24576, 24584, 0, 256, 0)
    assert e.value.arg == 9
    with pytest.raises(bto.BtoError) as e:     # no workspace
        bto.bto_csr_bicgk(4, 4, 3, 4096, 8192, 12288, 16384, 20480, 24576, 28672, 0, 0, 0)
    assert e.value.status == _lib.BTO_ERR_WORKSPACE and e.value.arg == 11
    with pytest.raises(bto.BtoError) as e:     # y overlapping x
        bto.bto_csr_atax(4, 4, 3, 4096, 8192, 12288, 1.0, 16384, 16392, 0, 256, 0)
    assert e.value.arg == 9


# ------------------------------------------------------------------ GPU


def _dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(device="cuda", dtype=dtype)


def _run_bicgk(m, n, rp, col, val, p, r):
    import torch
    d = [_dev(rp), _dev(col), _dev(val), _dev(p), _dev(r)]
    q = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device="cuda")
    s = torch.full((max(n, 1),), np.nan, dtype=torch.float64, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    bto.bto_csr_bicgk(m, n, len(col), d[0], d[1] if len(col) else None, d[2] if len(col) else None,
                      d[3] if n else None, d[4] if m else None, q if m else None, s if n else None, ws, 256)
    torch.cuda.synchronize()
    return q.cpu().numpy()[:m], s.cpu().numpy()[:n], ws


def _status(ws):
    import torch
    torch.cuda.synchronize()
    return int(ws[:4].view(torch.int32).cpu().numpy()[0])


CASES = [(1000, 800, 5), (3000, 2000, 40), (500, 3000, 150), (4099, 37, 3), (1, 1, 1), (0, 10, 3),
         (10, 0, 3), (200, 100, 0), (64, 64, 17)]


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,avg", CASES)
def test_csr_bicgk_matches_oracle(m, n, avg):
    from gpu_util import TOL64, relerr
    build.build()
    rp, col, val = synth.csr(7, 60, m, n, avg)
    p, r = synth.vector(7, 1, n), synth.vector(7, 2, m)
    q, s, ws = _run_bicgk(m, n, rp, col, val, p, r)
    rq, rs = O.csr_bicgk(m, n, rp, col, val, p, r)
    assert relerr(q, rq) <= TOL64 and relerr(s, rs) <= TOL64
    assert _status(ws) == _lib.BTO_OK
    q2, s2, _ = _run_bicgk(m, n, rp, col, val, p, r)
    assert np.array_equal(q, q2)           # row sums in a fixed order


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,avg", CASES)
def test_csr_atax_matches_oracle(m, n, avg):
    import torch
    from gpu_util import TOL64, relerr
    build.build()
    rp, col, val = synth.csr(8, 60, m, n, avg)
    x = synth.vector(8, 1, n)
    y = torch.full((max(n, 1),), np.nan, dtype=torch.float64, device="cuda")
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    d = [_dev(rp), _dev(col), _dev(val), _dev(x)]
    bto.bto_csr_atax(m, n, len(col), d[0], d[1] if len(col) else None, d[2] if len(col) else None, 0.75,
                     d[3] if n else None, y if n else None, ws, 256)
    got = y.cpu().numpy()[:n]
    assert relerr(got, O.csr_atax(m, n, 0.75, rp, col, val, x)) <= TOL64
    assert _status(ws) == _lib.BTO_OK


@pytest.mark.gpu
def test_csr_bad_indices_are_skipped_and_reported():
    """A column index outside [0, n) and a decreasing row pointer: the
    entries are skipped (never dereferenced), the rest is computed, and the
    status word reads BTO_ERR_INVALID_VALUE."""
    from gpu_util import TOL64, relerr
    build.build()
    m, n = 300, 200
    rp, col, val = synth.csr(9, 60, m, n, 6)
    bad = col.copy()
    bad[5] = n                 # out of range
    bad[11] = -3               # negative
    q, s, ws = _run_bicgk(m, n, rp, bad, val, synth.vector(9, 1, n), synth.vector(9, 2, m))
    assert _status(ws) == _lib.BTO_ERR_INVALID_VALUE
    v0 = val.copy()
    v0[[5, 11]] = 0.0
    c0 = bad.copy()
    c0[[5, 11]] = 0
    rq, rs = O.csr_bicgk(m, n, rp, c0, v0, synth.vector(9, 1, n), synth.vector(9, 2, m))
    assert relerr(q, rq) <= TOL64 and relerr(s, rs) <= TOL64
    # Row pointers that decrease, or run past nnz: clamped and reported.
    rp2 = rp.copy()
    rp2[50] = rp2[49] - 1 if rp2[49] > 0 else rp2[50]
    rp2[m] = len(col) + 1000
    q, s, ws = _run_bicgk(m, n, rp2, col, val, synth.vector(9, 1, n), synth.vector(9, 2, m))
    assert _status(ws) == _lib.BTO_ERR_INVALID_VALUE
    assert np.all(np.isfinite(q)) and np.all(np.isfinite(s))
