"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the fused BLAS sequences: it only turns
(seed, array id, element index) into numbers.  The generator is SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), used as a counter-based stream:

    key(seed, aid)     = fmix(seed * 2**32 + aid)                 (mod 2**64)
    u64(seed, aid, k)  = fmix(key + (k + 1) * GAMMA)              (mod 2**64)
    fmix(z)            : z ^= z >> 30; z *= M1; z ^= z >> 27; z *= M2; z ^= z >> 31

so u64(seed, aid, k) is the k-th output (0-based) of a SplitMix64 generator
whose state starts at key.  From it:

    uniform in [-1, 1): 2 * ((u64 >> 11) * 2**-53) - 1   (exact in FP64)
    integer in [-8, 8]: ((u64 >> 11) mod 17) - 8

A matrix element (i, j) of an m-by-n matrix uses k = i + j*m (the logical
column-major index, independent of the leading dimension); a vector element
i uses k = i.  The library exports a device-side fill with the same
definition (bto_fill_*), so inputs of several GiB can be generated in place.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

KIND_UNIFORM = 0   # U[-1, 1)
KIND_INTEGER = 1   # integers in [-8, 8]

# Array ids (the order the workloads list their operands).
GEMVER_IDS = dict(A=0, u1=1, v1=2, u2=3, v2=4, y=5, z=6)
COLSCALE_ID = 7


def _fmix(z):
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * M1
        z = z ^ (z >> np.uint64(27))
        z = z * M2
        z = z ^ (z >> np.uint64(31))
    return z


def key(seed, aid):
    s = (int(seed) << 32) + int(aid)
    return _fmix(np.array([s & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]


def u64(seed, aid, k):
    """Raw 64-bit outputs for counter values k (uint64 array)."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key(seed, aid) + (k + np.uint64(1)) * GAMMA
    return _fmix(z)


def values(seed, aid, k, kind=KIND_UNIFORM):
    """FP64 values for counter values k."""
    r = u64(seed, aid, k) >> np.uint64(11)
    if kind == KIND_UNIFORM:
        return 2.0 * (r.astype(np.float64) * 2.0 ** -53) - 1.0
    if kind == KIND_INTEGER:
        return (r % np.uint64(17)).astype(np.float64) - 8.0
    raise ValueError("unknown kind")


def vector(seed, aid, n, kind=KIND_UNIFORM, chunk=1 << 24):
    out = np.empty(int(n), dtype=np.float64)
    for s in range(0, int(n), chunk):
        e = min(int(n), s + chunk)
        out[s:e] = values(seed, aid, np.arange(s, e, dtype=np.uint64), kind)
    return out


def colscale(seed, n):
    """Per-column scale 10**(8u - 4), u in [0, 1) from array id 7 (host only)."""
    r = u64(seed, COLSCALE_ID, np.arange(int(n), dtype=np.uint64)) >> np.uint64(11)
    u = r.astype(np.float64) * 2.0 ** -53
    return np.power(10.0, 8.0 * u - 4.0)


def matrix(seed, aid, m, n, lda=None, kind=KIND_UNIFORM, scale=None, pad=np.nan):
    """m-by-n FP64 matrix, column-major with leading dimension lda.

    Returns an (lda, n) Fortran-ordered array; rows m..lda-1 hold `pad`.
    With `scale` (length n) column j is multiplied by scale[j].
    """
    m, n = int(m), int(n)
    lda = max(1, m) if lda is None else int(lda)
    a = np.full((lda, n), pad, dtype=np.float64, order="F")
    if m and n:
        for j0 in range(0, n, max(1, (1 << 24) // max(1, m))):
            j1 = min(n, j0 + max(1, (1 << 24) // max(1, m)))
            jj = np.arange(j0, j1, dtype=np.uint64)
            ii = np.arange(m, dtype=np.uint64)
            k = ii[:, None] + jj[None, :] * np.uint64(m)
            blk = values(seed, aid, k, kind)
            if scale is not None:
                blk = blk * scale[None, j0:j1]
            a[:m, j0:j1] = blk
    return a


def matrix_rows(seed, aid, m, n, rows, kind=KIND_UNIFORM, scale=None):
    """Rows `rows` (all n columns) of the m-by-n matrix, as a (len(rows), n) array."""
    rows = np.asarray(rows, dtype=np.uint64)
    jj = np.arange(int(n), dtype=np.uint64)
    k = rows[:, None] + jj[None, :] * np.uint64(m)
    v = values(seed, aid, k, kind)
    return v if scale is None else v * scale[None, :]


def matrix_cols(seed, aid, m, n, cols, kind=KIND_UNIFORM, scale=None):
    """Columns `cols` (all m rows) of the m-by-n matrix, as an (m, len(cols)) array."""
    cols = np.asarray(cols, dtype=np.uint64)
    ii = np.arange(int(m), dtype=np.uint64)
    k = ii[:, None] + cols[None, :] * np.uint64(m)
    v = values(seed, aid, k, kind)
    return v if scale is None else v * scale[None, np.asarray(cols, dtype=np.int64)]


def to_f32(a):
    """Round-to-nearest-even FP64 -> FP32 (numpy's cast is RNE)."""
    return np.asarray(a, dtype=np.float64).astype(np.float32)


def to_bf16_bits(a):
    """Round-to-nearest-even FP64 -> BF16, one rounding, as uint16 bit patterns.

    Finite inputs in the normal BF16 range only (the generators never leave it).
    """
    a = np.asarray(a, dtype=np.float64)
    b = a.view(np.uint64)
    # Round the 52-bit mantissa to 7 bits (RNE), carrying into the exponent.
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    with np.errstate(over="ignore"):
        r = (b + np.uint64(0x0FFFFFFFFFFF) + lsb) >> np.uint64(45)
    sign = (r >> np.uint64(18)) & np.uint64(1)
    exp = ((r >> np.uint64(7)) & np.uint64(0x7FF)).astype(np.int64)
    man = r & np.uint64(0x7F)
    e8 = exp - 1023 + 127
    zero = exp == 0
    e8 = np.where(zero, 0, e8)
    man = np.where(zero, np.uint64(0), man)
    if np.any((e8 <= 0) & ~zero) or np.any(e8 >= 255):
        raise ValueError("value outside the normal BF16 range")
    bits = (sign << np.uint64(15)) | (e8.astype(np.uint64) << np.uint64(7)) | man
    return bits.astype(np.uint16)


def bf16_bits_to_f64(bits):
    bits = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << np.uint32(16)
    return bits.view(np.float32).astype(np.float64)


def csr(seed, aid, m, n, avg_row):
    """A seeded m-by-n sparse matrix in compressed sparse rows.

    Row i holds u64(seed, aid, i) mod (2 avg_row + 1) entries (mean avg_row;
    none when n = 0); the entry at storage index k has column
    u64(seed, aid + 1, k) mod n and value U[-1, 1) from (seed, aid + 2, k).
    Columns are unsorted and may repeat within a row.  Returns (row_ptr
    int64[m + 1], col int32[nnz], val float64[nnz])."""
    m, n = int(m), int(n)
    if n == 0 or m == 0:
        lens = np.zeros(m, dtype=np.int64)
    else:
        lens = (u64(seed, aid, np.arange(m, dtype=np.uint64)) % np.uint64(2 * int(avg_row) + 1)).astype(np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    k = np.arange(nnz, dtype=np.uint64)
    col = (u64(seed, aid + 1, k) % np.uint64(max(n, 1))).astype(np.int32) if nnz else np.zeros(0, np.int32)
    val = values(seed, aid + 2, k) if nnz else np.zeros(0)
    return row_ptr, col, val
