"""Python face of the CPU oracle (plain C, FP64, unfused loop nests).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package; the library's product
path never does.

Matrices are numpy arrays of shape (ld, n) in Fortran (column-major) order;
the leading dimension is taken from the array (ld >= m, rows m..ld-1 are
never read or written).  Vectors are contiguous float64 arrays.  Every
function allocates and returns its outputs.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int64


def lib(path=None):
    """Load (building first if needed) the oracle library; `path` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


_par = None
PAR_NAMES = ("bicgk", "atax", "gemver", "gesummv", "dgemv", "dgemvt", "axpydot", "waxpby", "vadd")


class _ParLib:
    """The all-core build (bto_oracle_par.c) under the serial names, so that
    every function below takes it as L=...; routines it does not have are not
    reachable through it."""

    def __init__(self, cdll):
        serial = _bind_names()
        for k in PAR_NAMES:
            f = getattr(cdll, "oracle_par_" + k)
            f.argtypes = serial["oracle_" + k][0]
            f.restype = serial["oracle_" + k][1]
            setattr(self, "oracle_" + k, f)


def lib_par():
    """Load (building first if needed) the all-core oracle (OpenMP)."""
    global _par
    if _par is None:
        _par = _ParLib(ctypes.CDLL(_build.build_par()))
    return _par


def _bind_names():
    """{C name: (argtypes, restype)} of the oracle's exported routines."""
    d, i = ctypes.c_double, _I
    sig = _SIG(d, i)
    out = {}
    for name, args in sig.items():
        rt = ctypes.c_int if name in ("oracle_atax", "oracle_gemver", "oracle_gesummv", "oracle_dgemv",
                                      "oracle_dgemvt", "oracle_csr_atax",
                                      "oracle_band_bicgk", "oracle_band_atax") else (
            ctypes.c_double if name in ("oracle_dot2", "oracle_row_dot") else None)
        out[name] = (args, rt)
    return out


def _bind(L):
    for name, (args, rt) in _bind_names().items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = rt
    return L


def _SIG(d, i):
    return {
        "oracle_bicgk": [i, i, _D, i, _D, _D, _D, _D],
        "oracle_atax": [i, i, d, _D, i, _D, _D],
        "oracle_gemver": [i, i, d, d, _D, i, _D, _D, _D, _D, _D, _D, _D, i, _D, _D],
        "oracle_gesummv": [i, i, d, _D, i, d, _D, i, _D, _D],
        "oracle_dgemv": [i, i, d, _D, i, _D, d, _D, _D],
        "oracle_dgemvt": [i, i, d, d, _D, i, _D, _D, _D, _D],
        "oracle_axpydot": [i, d, _D, _D, _D, _D, _D],
        "oracle_axpydot_dot2": [i, d, _D, _D, _D, _D, _D],
        "oracle_waxpby": [i, d, _D, d, _D, _D],
        "oracle_vadd": [i, _D, _D, _D, _D],
        "oracle_dot2": [i, _D, _D],
        "oracle_bicgk_mrhs": [i, i, i, _D, i, _D, i, _D, i, _D, i, _D, i],
        "oracle_row_dot": [i, _D, _D],
        "oracle_csr_bicgk": [i, i, ctypes.c_void_p, ctypes.c_void_p, _D, _D, _D, _D, _D],
        "oracle_csr_atax": [i, i, d, ctypes.c_void_p, ctypes.c_void_p, _D, _D, _D],
        "oracle_band_bicgk": [ctypes.c_int, i, i, i, i, ctypes.c_int, _D, i, _D, _D, _D, _D],
        "oracle_band_atax": [ctypes.c_int, i, i, i, i, ctypes.c_int, d, _D, i, _D, _D],
    }


def _p(a):
    if a.size == 0:
        # A valid pointer for zero-length arrays (never dereferenced).
        a = np.zeros(1, dtype=np.float64)
        _p._keep.append(a)
    return a.ctypes.data_as(_D)


_p._keep = []


def _vec(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.ndim == 1
    return x


def _mat(A, m):
    A = np.asfortranarray(A, dtype=np.float64)
    assert A.ndim == 2
    ld = max(1, A.shape[0])
    assert A.shape[0] >= m or A.size == 0
    return A, ld


def _chk(rc):
    if rc != 0:
        raise MemoryError("oracle allocation failed")


def _csr(row_ptr, col, val):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    return rp, ci, v


def csr_bicgk(m, n, row_ptr, col, val, p, r, L=None):
    """Sparse BICGK on CSR arrays (row_ptr int64, col int32, val FP64)."""
    L = L or lib()
    rp, ci, v = _csr(row_ptr, col, val)
    p, r = _vec(p), _vec(r)
    q, s = np.empty(m), np.empty(n)
    L.oracle_csr_bicgk(m, n, rp.ctypes.data, ci.ctypes.data if ci.size else None, _p(v), _p(p), _p(r),
                       _p(q), _p(s))
    return q, s


def csr_atax(m, n, beta, row_ptr, col, val, x, L=None):
    """Sparse BATAX on CSR arrays."""
    L = L or lib()
    rp, ci, v = _csr(row_ptr, col, val)
    x = _vec(x)
    y = np.empty(n)
    _chk(L.oracle_csr_atax(m, n, beta, rp.ctypes.data, ci.ctypes.data if ci.size else None, _p(v), _p(x),
                           _p(y)))
    return y


STORE_FULL, STORE_BAND, STORE_PACKED = 0, 1, 2


def _band_args(storage, m, n, kl, ku, A, ld):
    """Checks a structured operand: A is the flat FP64 storage array (full:
    ld x n column-major; band: ld x n band array; packed: n (n + 1) / 2
    entries of a square triangle, kl = 0 upper or ku = 0 lower)."""
    assert m >= 0 and n >= 0 and 0 <= kl < 2 ** 40 and 0 <= ku < 2 ** 40
    A = np.ascontiguousarray(A, dtype=np.float64).ravel()
    if storage == STORE_FULL:
        assert ld >= max(1, m) and A.size >= (ld * (n - 1) + m if n and m else 0)
    elif storage == STORE_BAND:
        assert ld >= kl + ku + 1 and A.size >= (ld * n if m else 0)
    else:
        assert storage == STORE_PACKED and m == n and (kl == 0 or ku == 0)
        assert A.size >= n * (n + 1) // 2
    return kl, ku, A


def band_bicgk(storage, m, n, kl, ku, unit, A, ld, p, r, L=None):
    """BICGK on a banded or triangular matrix in full, band or packed storage."""
    L = L or lib()
    kl, ku, A = _band_args(storage, m, n, kl, ku, A, ld)
    p, r = _vec(p), _vec(r)
    q, s = np.empty(m), np.empty(n)
    _chk(L.oracle_band_bicgk(storage, m, n, kl, ku, int(unit), _p(A), max(int(ld), 1), _p(p), _p(r),
                             _p(q), _p(s)))
    return q, s


def band_atax(storage, m, n, kl, ku, unit, beta, A, ld, x, L=None):
    """BATAX on a banded or triangular matrix: y = beta A^T (A x)."""
    L = L or lib()
    kl, ku, A = _band_args(storage, m, n, kl, ku, A, ld)
    x = _vec(x)
    y = np.empty(n)
    _chk(L.oracle_band_atax(storage, m, n, kl, ku, int(unit), beta, _p(A), max(int(ld), 1), _p(x), _p(y)))
    return y


def bicgk(m, n, A, p, r, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    p, r = _vec(p), _vec(r)
    q, s = np.empty(m), np.empty(n)
    L.oracle_bicgk(m, n, _p(A), lda, _p(p), _p(r), _p(q), _p(s))
    return q, s


def atax(m, n, beta, A, x, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    x = _vec(x)
    y = np.empty(n)
    _chk(L.oracle_atax(m, n, beta, _p(A), lda, _p(x), _p(y)))
    return y


def gemver(m, n, alpha, beta, A, u1, v1, u2, v2, y, z, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    u1, v1, u2, v2, y, z = map(_vec, (u1, v1, u2, v2, y, z))
    B = np.zeros((max(1, m), n), order="F")
    x, w = np.empty(n), np.empty(m)
    _chk(L.oracle_gemver(m, n, alpha, beta, _p(A), lda, _p(u1), _p(v1), _p(u2), _p(v2),
                         _p(y), _p(z), _p(B), max(1, m), _p(x), _p(w)))
    return B[:m], x, w


def gesummv(m, n, alpha, A, beta, B, x, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    B, ldb = _mat(B, m)
    x = _vec(x)
    y = np.empty(m)
    _chk(L.oracle_gesummv(m, n, alpha, _p(A), lda, beta, _p(B), ldb, _p(x), _p(y)))
    return y


def dgemv(m, n, alpha, A, x, beta, y, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    x, y = _vec(x), _vec(y)
    z = np.empty(m)
    _chk(L.oracle_dgemv(m, n, alpha, _p(A), lda, _p(x), beta, _p(y), _p(z)))
    return z


def dgemvt(m, n, alpha, beta, A, y, z, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    y, z = _vec(y), _vec(z)
    x, w = np.empty(n), np.empty(m)
    _chk(L.oracle_dgemvt(m, n, alpha, beta, _p(A), lda, _p(y), _p(z), _p(x), _p(w)))
    return x, w


def axpydot(n, alpha, w, v, u, compensated=False, L=None):
    L = L or lib()
    w, v, u = map(_vec, (w, v, u))
    z = np.empty(n)
    r = ctypes.c_double(0.0)
    f = L.oracle_axpydot_dot2 if compensated else L.oracle_axpydot
    f(n, alpha, _p(w), _p(v), _p(u), _p(z), ctypes.byref(r))
    return z, r.value


def waxpby(n, alpha, x, beta, y, L=None):
    L = L or lib()
    x, y = _vec(x), _vec(y)
    w = np.empty(n)
    L.oracle_waxpby(n, alpha, _p(x), beta, _p(y), _p(w))
    return w


def vadd(n, w, y, z, L=None):
    L = L or lib()
    w, y, z = map(_vec, (w, y, z))
    x = np.empty(n)
    L.oracle_vadd(n, _p(w), _p(y), _p(z), _p(x))
    return x


def dot2(x, y, L=None):
    L = L or lib()
    x, y = _vec(x), _vec(y)
    return L.oracle_dot2(len(x), _p(x), _p(y))


def row_dot(row, p, L=None):
    L = L or lib()
    row, p = _vec(row), _vec(p)
    return L.oracle_row_dot(len(row), _p(row), _p(p))


def bicgk_mrhs(m, n, k, A, P, R, L=None):
    L = L or lib()
    A, lda = _mat(A, m)
    P = np.asfortranarray(P, dtype=np.float64)
    R = np.asfortranarray(R, dtype=np.float64)
    Q = np.zeros((max(1, m), k), order="F")
    S = np.zeros((max(1, n), k), order="F")
    L.oracle_bicgk_mrhs(m, n, k, _p(A), lda, _p(P), max(1, P.shape[0]), _p(R),
                        max(1, R.shape[0]), _p(Q), max(1, m), _p(S), max(1, n))
    return Q[:m], S[:n]
