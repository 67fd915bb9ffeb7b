"""Banded and triangular BICGK and BATAX (bto_band_*, bto_tri_*).

CPU (no GPU): the entry points reject bad arguments before any CUDA call,
with the 1-based position of the first bad one, and the workspace queries
answer.  GPU: every storage kind matches the oracle (which is pinned in
oracle_pins.py) within 1e-12 normwise on shapes that span several tiles with
ragged tails, bitwise on integer-valued inputs; storage slots outside the
band hold NaN and must not matter; results are bitwise reproducible; and the
benchmarked workloads (upper triangle n = 16384 in full and packed storage,
a band of 65 diagonals at 2^20 rows) are checked on sampled outputs."""
import numpy as np
import pytest
import torch

import band_util as BU
import oracle as O
import synth
import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import _lib, build

TOL = 1e-12


def _err(fn, *args):
    # stream 0 (the legacy default stream handle): no torch CUDA call on the CPU
    with pytest.raises(bto.BtoError) as e:
        fn(*args, 0)
    return e.value


# ------------------------------------------------------------------ CPU


def test_workspace_queries():
    build.build()
    a = bto.bto_band_workspace_bytes("bicgk", 1000, 900, 3, 5)
    b = bto.bto_band_workspace_bytes("atax", 1000, 900, 3, 5)
    assert a >= 256 and b >= a + 1000 * 8 and a % 256 == 0
    assert bto.bto_band_workspace_bytes("bicgk", 0, 0, 0, 0) == 256
    t = bto.bto_tri_workspace_bytes("bicgk", _lib.BTO_UPPER, 5000)
    assert t == bto.bto_band_workspace_bytes("bicgk", 5000, 5000, 0, 4999)
    with pytest.raises(bto.BtoError):
        bto.bto_band_workspace_bytes("gemver", 10, 10, 1, 1)
    with pytest.raises(bto.BtoError):
        bto.bto_band_workspace_bytes("bicgk", 10, 10, -1, 1)


def test_argument_validation_cpu():
    build.build()
    F, B, P = _lib.BTO_STORE_FULL, _lib.BTO_STORE_BAND, _lib.BTO_STORE_PACKED
    fake = 1 << 20   # never dereferenced: every call below fails validation first
    v = fake + 4096
    call = bto.bto_band_bicgk
    assert _err(call, 7, 10, 10, 1, 1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 1
    assert _err(call, F, -1, 10, 1, 1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 2
    assert _err(call, F, 10, 10, -2, 1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 4
    assert _err(call, F, 10, 10, 1, -1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 5
    assert _err(call, F, 10, 10, 1, 1, 2, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 6
    assert _err(call, F, 10, 10, 1, 1, 0, 0, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 7
    assert _err(call, F, 10, 10, 1, 1, 0, fake, 9, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 8
    assert _err(call, B, 10, 10, 1, 1, 0, fake, 2, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 8
    # packed: square, and exactly one of the two triangles
    assert _err(call, P, 10, 9, 0, 8, 0, fake, 1, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 2
    assert _err(call, P, 10, 10, 0, 5, 0, fake, 1, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 5
    assert _err(call, P, 10, 10, 2, 9, 0, fake, 1, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 4
    # misaligned / missing vectors, outputs overlapping inputs
    assert _err(call, F, 10, 10, 1, 1, 0, fake, 10, v + 1, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 9
    assert _err(call, F, 10, 10, 1, 1, 0, fake, 10, v, v + 800, v + 1600, v + 1600, v + 8192, 1 << 20).arg == 11
    assert _err(call, F, 10, 10, 1, 1, 0, fake, 10, v, v + 800, fake + 8, v + 2400, v + 8192, 1 << 20).arg == 11
    # workspace too small / misaligned
    e = _err(call, F, 10, 10, 1, 1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 16)
    assert e.arg == 13 and e.status == _lib.BTO_ERR_WORKSPACE
    e = _err(call, F, 10, 10, 1, 1, 0, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192 + 8, 1 << 20)
    assert e.arg == 13
    # BATAX and the triangular forms
    assert _err(bto.bto_band_atax, F, 10, 10, 1, 1, 0, 1.0, fake, 10, v, v, v + 8192, 1 << 20).arg == 11
    assert _err(bto.bto_band_atax, F, 10, 10, 1, 1, 0, 1.0, fake, 10, v, v + 800, v + 8192, 8).arg == 12
    assert _err(bto.bto_tri_bicgk, 2, 0, 0, 10, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 1
    assert _err(bto.bto_tri_bicgk, 0, 3, 0, 10, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 2
    assert _err(bto.bto_tri_bicgk, 0, 0, 2, 10, fake, 10, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 3
    assert _err(bto.bto_tri_bicgk, 0, 0, 0, 10, fake, 9, v, v + 800, v + 1600, v + 2400, v + 8192, 1 << 20).arg == 6
    assert _err(bto.bto_tri_atax, 1, 0, 1, 10, 1.0, fake, 0, v, v, v + 8192, 1 << 20).arg == 9
    assert _err(bto.bto_tri_atax, 1, 0, 1, 10, 1.0, fake, 0, v, v + 800, v + 8192, 8).arg == 10


# ------------------------------------------------------------------ GPU

# (m, n, kl, ku): several tiles of 128 columns and of 32..256 band rows,
# ragged tails, bands wider than the matrix, one-sided bands, a diagonal.
SHAPES = [(300, 257, 5, 9), (1000, 700, 0, 699), (700, 1000, 699, 0), (2000, 1900, 300, 40),
          (5000, 5000, 1, 1), (4097, 4097, 32, 32), (50, 40, 100, 100), (129, 131, 0, 0),
          (3, 1000, 1, 600), (1000, 3, 600, 1), (640, 640, 63, 64), (777, 513, 200, 250)]
TRI = [(n, uplo) for n in (1, 2, 33, 129, 300, 1029) for uplo in (0, 1)]


def _call_band(storage, m, n, kl, ku, unit, D, p, r, beta=1.5, ld=None):
    A, ld = BU.store(D, storage, kl, ku, ld)
    dA = torch.from_numpy(A).cuda()
    dp, dr = torch.from_numpy(p).cuda(), torch.from_numpy(r).cuda()
    q = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    s = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    y = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    nb = bto.bto_band_workspace_bytes("atax", m, n, kl, ku)
    wk = torch.full((nb,), 0xA5, dtype=torch.uint8, device="cuda")
    bto.bto_band_bicgk(storage, m, n, kl, ku, unit, dA, ld, dp, dr, q, s, wk, nb, None)
    bto.bto_band_atax(storage, m, n, kl, ku, unit, beta, dA, ld, dp, y, wk, nb, None)
    torch.cuda.synchronize()
    assert bto.bto_device_status(wk) == 0
    return A, ld, q.cpu().numpy(), s.cpu().numpy(), y.cpu().numpy()


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.gpu
@pytest.mark.parametrize("storage", [BU.FULL, BU.BAND])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_kl%d_ku%d" % s)
def test_band_parity(shape, storage):
    build.build()
    m, n, kl, ku = shape
    D = BU.dense(7, 1, m, n, kl, ku)
    p, r = synth.vector(7, 2, n), synth.vector(7, 3, m)
    for unit in (0, 1):
        A, ld, q, s, y = _call_band(storage, m, n, kl, ku, unit, D, p, r)
        qo, so = O.band_bicgk(storage, m, n, kl, ku, unit, A, ld, p, r)
        yo = O.band_atax(storage, m, n, kl, ku, unit, 1.5, A, ld, p)
        assert _rel(q, qo) < TOL and _rel(s, so) < TOL and _rel(y, yo) < TOL, (shape, unit)


@pytest.mark.gpu
@pytest.mark.parametrize("packed", [0, 1])
@pytest.mark.parametrize("n,uplo", TRI)
def test_triangular_parity(n, uplo, packed):
    build.build()
    kl, ku = (0, n - 1) if uplo == 0 else (n - 1, 0)
    D = BU.dense(8, n, n, n, kl, ku)
    p, r = synth.vector(8, 2, n), synth.vector(8, 3, n)
    A, ld = (BU.store_packed(D, uplo == 0), 1) if packed else BU.store_full(D, kl, ku)
    dA = torch.from_numpy(A).cuda()
    dp, dr = torch.from_numpy(p).cuda(), torch.from_numpy(r).cuda()
    nb = bto.bto_tri_workspace_bytes("atax", uplo, n)
    wk = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = BU.PACKED if packed else BU.FULL
    for unit in (0, 1):
        q = torch.empty(n, dtype=torch.float64, device="cuda")
        s, y = torch.empty_like(q), torch.empty_like(q)
        bto.bto_tri_bicgk(uplo, unit, packed, n, dA, ld, dp, dr, q, s, wk, nb, None)
        bto.bto_tri_atax(uplo, unit, packed, n, -0.75, dA, ld, dp, y, wk, nb, None)
        torch.cuda.synchronize()
        qo, so = O.band_bicgk(st, n, n, kl, ku, unit, A, ld, p, r)
        yo = O.band_atax(st, n, n, kl, ku, unit, -0.75, A, ld, p)
        assert _rel(q.cpu().numpy(), qo) < TOL and _rel(s.cpu().numpy(), so) < TOL, (n, uplo, unit)
        assert _rel(y.cpu().numpy(), yo) < TOL, (n, uplo, unit)


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [(300, 257, 5, 9), (1029, 1029, 0, 1028), (1029, 1029, 1028, 0),
                                   (4097, 4097, 32, 32), (2000, 1900, 300, 40)])
def test_integer_exact_and_reproducible(shape):
    build.build()
    m, n, kl, ku = shape
    D = BU.dense(9, 1, m, n, kl, ku, kind=synth.KIND_INTEGER)
    p, r = synth.vector(9, 2, n, synth.KIND_INTEGER), synth.vector(9, 3, m, synth.KIND_INTEGER)
    A, ld, q, s, y = _call_band(BU.BAND, m, n, kl, ku, 0, D, p, r, beta=2.0)
    qo, so = O.band_bicgk(BU.BAND, m, n, kl, ku, 0, A, ld, p, r)
    yo = O.band_atax(BU.BAND, m, n, kl, ku, 0, 2.0, A, ld, p)
    assert np.array_equal(q, qo) and np.array_equal(s, so) and np.array_equal(y, yo)
    # floating-point values: two runs agree bitwise
    D = BU.dense(9, 2, m, n, kl, ku)
    p, r = synth.vector(9, 4, n), synth.vector(9, 5, m)
    a1 = _call_band(BU.FULL, m, n, kl, ku, 0, D, p, r)
    a2 = _call_band(BU.FULL, m, n, kl, ku, 0, D, p, r)
    for u, v in zip(a1[2:], a2[2:]):
        assert np.array_equal(u, v)


@pytest.mark.gpu
def test_nonfinite_outside_band_and_empty():
    build.build()
    n = 700
    D = BU.dense(10, 1, n, n, 2, 3)
    p, r = synth.vector(10, 2, n), synth.vector(10, 3, n)
    p[400] = np.inf
    r[100] = np.nan
    A, ld, q, s, y = _call_band(BU.BAND, n, n, 2, 3, 0, D, p, r)
    qo, so = O.band_bicgk(BU.BAND, n, n, 2, 3, 0, A, ld, p, r)
    # rows whose band misses column 400 and columns whose band misses row 100 stay finite
    fin_q, fin_s = np.isfinite(qo), np.isfinite(so)
    assert np.array_equal(np.isfinite(q), fin_q) and np.array_equal(np.isfinite(s), fin_s)
    assert fin_q.sum() == n - 6 and fin_s.sum() == n - 6
    assert _rel(q[fin_q], qo[fin_q]) < TOL and _rel(s[fin_s], so[fin_s]) < TOL
    # empty sizes: outputs are zero-length or zero sums
    for (m, k) in ((0, 5), (5, 0), (0, 0)):
        D = np.zeros((m, k))
        _, _, q, s, y = _call_band(BU.FULL, m, k, 1, 1, 0, D, np.ones(k), np.ones(m))
        assert np.array_equal(q, np.zeros(m)) and np.array_equal(s, np.zeros(k)) and np.array_equal(y, np.zeros(k))


def _samples(n, k=48, seed=5):
    return np.unique(np.concatenate([[0, 1, n - 2, n - 1, n // 2],
                                     ((synth.vector(seed, 77, k) * 0.5 + 0.5) * (n - 1))]).astype(np.int64))


@pytest.mark.gpu
@pytest.mark.parametrize("packed", [0, 1])
def test_triangle_n16384_sampled(packed):
    """The benchmarked triangle: upper, n = 16384.  Full storage is the
    synthetic n x n matrix (array id 0; the entries below the diagonal are
    never read); packed storage is the generator's stream itself, entry k of
    the packed array being value k of array id 0, so A(i, j) (i <= j) is value
    j (j + 1) / 2 + i."""
    build.build()
    n, seed = 16384, 1
    p, r = synth.vector(seed, 1, n), synth.vector(seed, 2, n)
    if packed:
        npk = n * (n + 1) // 2
        dA = torch.empty(npk, dtype=torch.float64, device="cuda")
        bto.bto_fill_f64(seed, 0, 0, npk, 1, 0, dA, npk, None)
        ld = 1
    else:
        dA = torch.empty(n * n, dtype=torch.float64, device="cuda")
        bto.bto_fill_f64(seed, 0, 0, n, n, 0, dA, n, None)
        ld = n
    nb = bto.bto_tri_workspace_bytes("atax", 0, n)
    wk = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dp, dr = torch.from_numpy(p).cuda(), torch.from_numpy(r).cuda()
    q, s, y = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    bto.bto_tri_bicgk(0, 0, packed, n, dA, ld, dp, dr, q, s, wk, nb, None)
    bto.bto_tri_atax(0, 0, packed, n, 1.0, dA, ld, dp, y, wk, nb, None)
    torch.cuda.synchronize()
    q, s, y = q.cpu().numpy(), s.cpu().numpy(), y.cpu().numpy()
    I, J = _samples(n), _samples(n, seed=6)
    if packed:
        jj = np.arange(n, dtype=np.uint64)
        RA = np.stack([synth.values(seed, 0, jj * (jj + np.uint64(1)) // np.uint64(2) + np.uint64(i)) for i in I])
        CA = np.stack([synth.values(seed, 0, np.uint64(j * (j + 1) // 2) + jj) for j in J], axis=1)
    else:
        RA = synth.matrix_rows(seed, 0, n, n, I)
        CA = synth.matrix_cols(seed, 0, n, n, J)
    for k, i in enumerate(I):
        # row i of the upper triangle: columns i..n-1, as a 1 x (n - i) band
        qo, _ = O.band_bicgk(BU.FULL, 1, n - i, 0, n - i - 1, 0, RA[k, i:], 1, p[i:], r[i:i + 1])
        assert abs(q[i] - qo[0]) <= TOL * max(abs(qo[0]), np.abs(RA[k, i:]) @ np.abs(p[i:])), i
    for k, j in enumerate(J):
        _, so = O.band_bicgk(BU.FULL, j + 1, 1, j, 0, 0, CA[:j + 1, k], j + 1, p[j:j + 1], r[:j + 1])
        assert abs(s[j] - so[0]) <= TOL * max(abs(so[0]), np.abs(CA[:j + 1, k]) @ np.abs(r[:j + 1])), j
    # BATAX: y = A^T (A x) with t = A x from the oracle on full rows would need
    # every row; check the property that holds at any size instead:
    # x^T y = |A x|^2 >= 0, against the t of the BICGK call above (q = A p).
    tq = float(q @ q)
    assert abs(float(p @ y) - tq) <= 1e-11 * tq


@pytest.mark.gpu
def test_band_2e20_sampled():
    """The benchmarked band: m = n = 2^20, kl = ku = 32, band storage
    (ld = 65) filled by the device generator as a 65 x n matrix (array id 0)."""
    build.build()
    n, kl, ku, seed = 1 << 20, 32, 32, 11
    ld = kl + ku + 1
    dA = torch.empty(ld * n, dtype=torch.float64, device="cuda")
    bto.bto_fill_f64(seed, 0, 0, ld, n, 0, dA, ld, None)
    p, r = synth.vector(seed, 1, n), synth.vector(seed, 2, n)
    nb = bto.bto_band_workspace_bytes("atax", n, n, kl, ku)
    wk = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dp, dr = torch.from_numpy(p).cuda(), torch.from_numpy(r).cuda()
    q, s, y = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    bto.bto_band_bicgk(BU.BAND, n, n, kl, ku, 0, dA, ld, dp, dr, q, s, wk, nb, None)
    bto.bto_band_atax(BU.BAND, n, n, kl, ku, 0, 0.5, dA, ld, dp, y, wk, nb, None)
    torch.cuda.synchronize()
    q, s, y = q.cpu().numpy(), s.cpu().numpy(), y.cpu().numpy()
    # A window of rows and columns around each sample holds every entry they
    # touch: run the oracle on that sub-band (band storage of the window).
    for c in _samples(n):
        j0, j1 = max(0, c - 2 * ld), min(n, c + 2 * ld)
        idx = (np.arange(ld)[:, None] + np.arange(j0, j1)[None, :] * ld).ravel(order="F")
        AB = synth.values(seed, 0, idx.astype(np.uint64))
        # sub-matrix rows/cols [j0, j1): its band storage is the same slice
        w = j1 - j0
        qo, so = O.band_bicgk(BU.BAND, w, w, kl, ku, 0, AB, ld, p[j0:j1], r[j0:j1])
        # interior rows/columns of the window have their whole band inside it
        lo, hi = (c - j0) - 8, (c - j0) + 8
        sl = slice(max(0, lo) if j0 == 0 else max(ld, lo), min(w, hi) if j1 == n else min(w - ld, hi))
        assert _rel(q[j0:j1][sl], qo[sl]) < TOL and _rel(s[j0:j1][sl], so[sl]) < TOL, c
    tq = float(q @ q)
    assert abs(float(p @ y) - 0.5 * tq) <= 1e-11 * 0.5 * tq
