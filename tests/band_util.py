"""Banded and triangular test operands (test infrastructure, no GPU).

A structured matrix is described by its shape m x n and its band: kl
sub-diagonals and ku super-diagonals (A(i, j) = 0 unless
j - ku <= i <= j + kl).  An upper triangle is kl = 0, ku = n - 1; a lower
one ku = 0, kl = m - 1.  These helpers build the dense matrix and its three
stored forms from the dense one by plain element loops, with NaN in every
storage slot the band does not use, so a kernel or oracle that reads outside
the band shows it.
"""
import numpy as np

import synth

FULL, BAND, PACKED = 0, 1, 2


def in_band(m, n, kl, ku):
    """Boolean m x n mask of the band."""
    i = np.arange(m)[:, None]
    j = np.arange(n)[None, :]
    return (i >= j - ku) & (i <= j + kl)


def dense(seed, aid, m, n, kl, ku, kind=synth.KIND_UNIFORM):
    """Dense FP64 matrix with synthetic values inside the band, 0 outside."""
    A = synth.matrix(seed, aid, m, n, kind=kind) if m and n else np.zeros((m, n))
    return np.where(in_band(m, n, kl, ku), A, 0.0)


def store_full(D, kl, ku, ld=None):
    """Column-major full storage (ld >= m) with NaN outside the band."""
    m, n = D.shape
    ld = ld or max(1, m)
    S = np.full((ld, n), np.nan, order="F")
    mask = in_band(m, n, kl, ku)
    S[:m][mask] = D[mask]
    return S.ravel(order="F"), ld


def store_band(D, kl, ku, ld=None):
    """Band storage: A(i, j) at row ku + i - j of column j, ld >= kl + ku + 1."""
    m, n = D.shape
    ld = ld or kl + ku + 1
    S = np.full(ld * n, np.nan)
    for j in range(n):
        for i in range(max(0, j - ku), min(m, j + kl + 1)):
            S[(ku + i - j) + j * ld] = D[i, j]
    return S, ld


def store_packed(D, upper):
    """Packed square triangle, column after column (upper: rows 0..j of
    column j; lower: rows j..n-1)."""
    n = D.shape[0]
    out = []
    for j in range(n):
        rows = range(0, j + 1) if upper else range(j, n)
        out.extend(D[i, j] for i in rows)
    return np.array(out, dtype=np.float64)


def store(D, storage, kl, ku, ld=None):
    """(flat storage, ld) of D in the given storage kind."""
    if storage == FULL:
        return store_full(D, kl, ku, ld)
    if storage == BAND:
        return store_band(D, kl, ku, ld)
    return store_packed(D, kl == 0), 1
