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
    nb = bto.bto_csr_workspace_bytes("bicgk", m, n, len(col))
    ws = torch.full((nb,), 0xA5, dtype=torch.uint8, device="cuda")
    bto.bto_csr_bicgk(m, n, len(col), d[0], d[1] if len(col) else None, d[2] if len(col) else None,
                      d[3] if n else None, d[4] if m else None, q if m else None, s if n else None, ws, nb)
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
    nb = bto.bto_csr_workspace_bytes("atax", m, n, len(col))
    ws = torch.full((nb,), 0xA5, dtype=torch.uint8, device="cuda")
    d = [_dev(rp), _dev(col), _dev(val), _dev(x)]
    bto.bto_csr_atax(m, n, len(col), d[0], d[1] if len(col) else None, d[2] if len(col) else None, 0.75,
                     d[3] if n else None, y if n else None, ws, nb)
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


def _structured_csr(lengths, n, seed):
    """CSR arrays with the given row lengths (columns and values seeded)."""
    rp = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    nnz = int(rp[-1])
    col = (synth.u64(seed, 90, np.arange(nnz, dtype=np.uint64)) % np.uint64(n)).astype(np.int32)
    val = synth.vector(seed, 91, nnz)
    return rp, col, val


# Row lengths that put row ends on lane (8-entry) and unit (256-entry)
# boundaries, empty rows at those boundaries, in runs and at the end, rows
# that span many units, and a single row holding everything.
PATTERNS = {
    "boundaries": [8, 0, 8, 0, 0, 248, 256, 0, 1, 7, 0, 8, 240, 0, 0, 512, 3, 0, 0],
    "long_rows": [0, 3, 5000, 0, 1, 2560, 7, 0, 0],
    "one_row": [12345],
    "empties_first": [0] * 40 + [300, 0, 5] + [0] * 9,
    "mixed": list(np.tile([0, 1, 2, 3, 17, 31, 32, 33, 255, 256, 257, 0], 20)),
}


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(PATTERNS))
def test_csr_row_patterns(name):
    """Rows crossing lane and unit boundaries, empty rows everywhere, long
    rows spanning many units: q and t bitwise reproducible and <= 1e-12 vs
    the oracle; the unaligned-pointer path (val and col one element off a
    16-byte boundary) gives the same row sums bitwise."""
    import torch
    from gpu_util import TOL64, relerr
    build.build()
    lengths = PATTERNS[name]
    m, n = len(lengths), 777
    rp, col, val = _structured_csr(lengths, n, 12)
    nnz = len(col)
    p, r = synth.vector(12, 1, n), synth.vector(12, 2, m)
    q, s, ws = _run_bicgk(m, n, rp, col, val, p, r)
    rq, rs = O.csr_bicgk(m, n, rp, col, val, p, r)
    assert _status(ws) == _lib.BTO_OK
    assert relerr(q, rq) <= TOL64 and relerr(s, rs) <= TOL64
    assert np.all(q[np.diff(rp) == 0] == 0.0)
    # unaligned entry arrays: one element into larger buffers
    dcol = torch.from_numpy(np.concatenate([[0], col]).astype(np.int32)).cuda()
    dval = torch.from_numpy(np.concatenate([[0.0], val])).cuda()
    q2 = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    s2 = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    nb = bto.bto_csr_workspace_bytes("bicgk", m, n, nnz)
    w2 = torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda")
    bto.bto_csr_bicgk(m, n, nnz, _dev(rp), dcol.data_ptr() + 4, dval.data_ptr() + 8, _dev(p), _dev(r), q2, s2,
                      w2, nb)
    assert _status(w2) == _lib.BTO_OK
    assert np.array_equal(q, q2.cpu().numpy())
    # BATAX on the same pattern
    y = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    nb = bto.bto_csr_workspace_bytes("atax", m, n, nnz)
    w3 = torch.full((nb,), 0x5A, dtype=torch.uint8, device="cuda")
    bto.bto_csr_atax(m, n, nnz, _dev(rp), _dev(col), _dev(val), -1.25, _dev(p), y, w3, nb)
    assert _status(w3) == _lib.BTO_OK
    assert relerr(y.cpu().numpy(), O.csr_atax(m, n, -1.25, rp, col, val, p)) <= TOL64


def test_csr_workspace_query():
    build.build()
    a = bto.bto_csr_workspace_bytes("bicgk", 1000, 1000, 256 * 1000)
    b = bto.bto_csr_workspace_bytes("atax", 1000, 1000, 256 * 1000)
    assert a % 256 == 0 and a >= 256 + 3 * 8 * 1000 and b >= a + 8 * 1000
    assert bto.bto_csr_workspace_bytes("bicgk", 0, 0, 0) >= 256
    with pytest.raises(bto.BtoError):
        bto.bto_csr_workspace_bytes("gemver", 1, 1, 1)
