"""Pins for the oracle: checks that tie it to something other than itself.

Each pin is a function (L) -> None that raises AssertionError on failure, where
L is a loaded oracle library (the real one, or a mutant built by the mutation
test).  The pins are:
  * hand-worked examples under tests/golden/ (values computed by hand);
  * integer-valued inputs, where every FP64 partial sum is exact, compared
    bitwise with exact int64 arithmetic (brute force);
  * closed forms (all-ones and rank-1 matrices), the adjoint identity of
    BICGK, a second formula for GEMVER that never forms B, and special cases
    that reduce to an exact zero or to the input;
  * the Dot2 error bound of Ogita, Rump and Oishi against an exact rational sum;
  * for the sparse (CSR) definitions: a hand-worked example, integer-valued
    inputs against exact products of the densified matrix, the identity;
  * for the banded and triangular definitions: hand-worked examples in every
    storage kind (with NaN in the slots outside the band), integer-valued
    inputs against exact products of the dense matrix, prefix/suffix sums of
    an all-ones triangle, the second difference of a tridiagonal matrix, the
    adjoint identity, and bitwise agreement of the three storage kinds.
"""
from fractions import Fraction

import numpy as np

import band_util as BU
import oracle as O
import synth
from golden_io import colmajor, load


def _ints(seed, aid, n):
    return synth.vector(seed, aid, n, synth.KIND_INTEGER)


def _imat(seed, aid, m, n, lda=None):
    return synth.matrix(seed, aid, m, n, lda=lda, kind=synth.KIND_INTEGER)


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


# ---------------------------------------------------------------- golden
def pin_golden(L):
    g, e = load("bicgk_2x3.txt")
    q, s = O.bicgk(g["m"], g["n"], colmajor(g["A"], g["m"], g["n"]), g["p"], g["r"], L=L)
    assert np.array_equal(q, e["q"]) and np.array_equal(s, e["s"]), (q, s)

    g, e = load("atax_2x3.txt")
    y = O.atax(g["m"], g["n"], g["beta"], colmajor(g["A"], g["m"], g["n"]), g["x"], L=L)
    assert np.array_equal(y, e["y"]), y

    g, e = load("gemver_2x2.txt")
    B, x, w = O.gemver(g["m"], g["n"], g["alpha"], g["beta"], colmajor(g["A"], g["m"], g["n"]),
                       g["u1"], g["v1"], g["u2"], g["v2"], g["y"], g["z"], L=L)
    assert np.array_equal(B.ravel(order="F"), e["B"]), B
    assert np.array_equal(x, e["x"]) and np.array_equal(w, e["w"]), (x, w)

    g, e = load("gesummv_2x2.txt")
    y = O.gesummv(g["m"], g["n"], g["alpha"], colmajor(g["A"], g["m"], g["n"]), g["beta"],
                  colmajor(g["B"], g["m"], g["n"]), g["x"], L=L)
    assert np.array_equal(y, e["y"]), y

    g, e = load("dgemv_2x3.txt")
    z = O.dgemv(g["m"], g["n"], g["alpha"], colmajor(g["A"], g["m"], g["n"]), g["x"],
                g["beta"], g["y"], L=L)
    assert np.array_equal(z, e["z"]), z

    g, e = load("dgemvt_2x3.txt")
    x, w = O.dgemvt(g["m"], g["n"], g["alpha"], g["beta"], colmajor(g["A"], g["m"], g["n"]),
                    g["y"], g["z"], L=L)
    assert np.array_equal(x, e["x"]) and np.array_equal(w, e["w"]), (x, w)

    g, e = load("axpydot_4.txt")
    for comp in (False, True):
        z, r = O.axpydot(g["n"], g["alpha"], g["w"], g["v"], g["u"], compensated=comp, L=L)
        assert np.array_equal(z, e["z"]) and r == e["r"][0], (z, r)

    g, e = load("waxpby_3.txt")
    w = O.waxpby(g["n"], g["alpha"], g["x"], g["beta"], g["y"], L=L)
    assert np.array_equal(w, e["w"]), w

    for name in ("vadd_3.txt", "vadd_order.txt"):
        g, e = load(name)
        x = O.vadd(g["n"], g["w"], g["y"], g["z"], L=L)
        assert np.array_equal(x, e["x"]), (name, x)


# ---------------------------------------------------------------- exact integers
M, N = 37, 53   # ragged, non-square


def pin_integer_exact(L):
    A = _imat(5, 0, M, N, lda=M + 3)
    Ai = A[:M].astype(np.int64)
    p, r = _ints(5, 1, N), _ints(5, 2, M)
    q, s = O.bicgk(M, N, A, p, r, L=L)
    assert np.array_equal(q, (Ai @ p.astype(np.int64)).astype(float))
    assert np.array_equal(s, (Ai.T @ r.astype(np.int64)).astype(float))

    x = _ints(5, 3, N)
    y = O.atax(M, N, 3.0, A, x, L=L)
    assert np.array_equal(y, (3 * (Ai.T @ (Ai @ x.astype(np.int64)))).astype(float))

    u1, u2, yv = _ints(5, 4, M), _ints(5, 5, M), _ints(5, 6, M)
    v1, v2, zv = _ints(5, 7, N), _ints(5, 8, N), _ints(5, 9, N)
    B, xg, wg = O.gemver(M, N, 2.0, -3.0, A, u1, v1, u2, v2, yv, zv, L=L)
    Bi = Ai + np.outer(u1, v1).astype(np.int64) + np.outer(u2, v2).astype(np.int64)
    xi = -3 * (Bi.T @ yv.astype(np.int64)) + zv.astype(np.int64)
    wi = 2 * (Bi @ xi)
    assert np.array_equal(B, Bi.astype(float))
    assert np.array_equal(xg, xi.astype(float)) and np.array_equal(wg, wi.astype(float))

    Bm = _imat(5, 10, M, N)
    yy = O.gesummv(M, N, 2.0, A, -1.0, Bm, x, L=L)
    assert np.array_equal(yy, (2 * (Ai @ x.astype(np.int64))
                               - Bm.astype(np.int64) @ x.astype(np.int64)).astype(float))

    yd = _ints(5, 11, M)
    z = O.dgemv(M, N, 3.0, A, x, -2.0, yd, L=L)
    assert np.array_equal(z, (3 * (Ai @ x.astype(np.int64)) - 2 * yd.astype(np.int64)).astype(float))

    zt = _ints(5, 12, N)
    xt, wt = O.dgemvt(M, N, -1.0, 2.0, A, yd, zt, L=L)
    xti = 2 * (Ai.T @ yd.astype(np.int64)) + zt.astype(np.int64)
    assert np.array_equal(xt, xti.astype(float))
    assert np.array_equal(wt, (-(Ai @ xti)).astype(float))

    n = 1001
    w, v, u = _ints(6, 0, n), _ints(6, 1, n), _ints(6, 2, n)
    for comp in (False, True):
        zz, rr = O.axpydot(n, 3.0, w, v, u, compensated=comp, L=L)
        zi = w.astype(np.int64) - 3 * v.astype(np.int64)
        assert np.array_equal(zz, zi.astype(float)) and rr == float(zi @ u.astype(np.int64))
    ww = O.waxpby(n, 2.0, w, -3.0, v, L=L)
    assert np.array_equal(ww, (2 * w.astype(np.int64) - 3 * v.astype(np.int64)).astype(float))
    xx = O.vadd(n, w, v, u, L=L)
    assert np.array_equal(xx, (w.astype(np.int64) + v.astype(np.int64) + u.astype(np.int64)).astype(float))


# ---------------------------------------------------------------- closed forms
def pin_closed_forms(L):
    m, n = 29, 41
    p, r, x = synth.vector(7, 1, n), synth.vector(7, 2, m), synth.vector(7, 3, n)
    ones = np.ones((m, n), order="F")
    q, s = O.bicgk(m, n, ones, p, r, L=L)
    assert _rel(q, np.full(m, np.sum(p))) < 1e-14 and _rel(s, np.full(n, np.sum(r))) < 1e-14
    y = O.atax(m, n, 1.0, ones, x, L=L)
    assert _rel(y, np.full(n, m * np.sum(x))) < 1e-14
    # rank-1 A = a b^T
    a, b = synth.vector(7, 4, m), synth.vector(7, 5, n)
    R1 = np.asfortranarray(np.outer(a, b))
    q, s = O.bicgk(m, n, R1, p, r, L=L)
    assert _rel(q, a * np.dot(b, p)) < 1e-13 and _rel(s, b * np.dot(a, r)) < 1e-13
    y = O.atax(m, n, 0.5, R1, x, L=L)
    assert _rel(y, 0.5 * b * np.dot(a, a) * np.dot(b, x)) < 1e-13
    z = O.dgemv(m, n, 2.0, R1, x, -1.0, r, L=L)
    assert _rel(z, 2.0 * a * np.dot(b, x) - r) < 1e-13
    # GEMVER with A = u = v = 1: B = 3, x_j = 3 beta sum(y) + z_j, w_i = 3 alpha sum(x)
    o_m, o_n = np.ones(m), np.ones(n)
    yv, zv = synth.vector(7, 6, m), synth.vector(7, 7, n)
    B, xg, wg = O.gemver(m, n, 1.5, 1.2, ones, o_m, o_n, o_m, o_n, yv, zv, L=L)
    assert np.all(B == 3.0)
    assert _rel(xg, 3 * 1.2 * np.sum(yv) + zv) < 1e-14
    assert _rel(wg, np.full(m, 3 * 1.5 * np.sum(xg))) < 1e-14


def pin_identities(L):
    m, n = 61, 47
    A = synth.matrix(8, 0, m, n, lda=m + 5)
    Am = A[:m]
    p, r = synth.vector(8, 1, n), synth.vector(8, 2, m)
    q, s = O.bicgk(m, n, A, p, r, L=L)
    # adjoint identity r^T (A p) = (A^T r)^T p
    scale = np.abs(r) @ np.abs(Am) @ np.abs(p)
    assert abs(np.dot(r, q) - np.dot(s, p)) < 1e-13 * scale
    # GEMVER without forming B:
    #   x = beta (A^T y + v1 (u1.y) + v2 (u2.y)) + z,  w = alpha (A x + u1 (v1.x) + u2 (v2.x))
    u1, u2, yv = (synth.vector(8, k, m) for k in (3, 4, 5))
    v1, v2, zv = (synth.vector(8, k, n) for k in (6, 7, 8))
    al, be = 1.5, 1.2
    B, xg, wg = O.gemver(m, n, al, be, A, u1, v1, u2, v2, yv, zv, L=L)
    x2 = be * (Am.T @ yv + v1 * np.dot(u1, yv) + v2 * np.dot(u2, yv)) + zv
    assert _rel(xg, x2) < 1e-13
    w2 = al * (Am @ xg + u1 * np.dot(v1, xg) + u2 * np.dot(v2, xg))
    assert _rel(wg, w2) < 1e-13
    assert _rel(B, Am + np.outer(u1, v1) + np.outer(u2, v2)) < 1e-15
    # DGEMVT: the second statement uses the new x
    xt, wt = O.dgemvt(m, n, 2.0, -0.5, A, yv, zv, L=L)
    assert _rel(xt, -0.5 * (Am.T @ yv) + zv) < 1e-13
    assert _rel(wt, 2.0 * (Am @ xt)) < 1e-13
    # GESUMMV: B = A gives (alpha + beta) A x ; B = -A with alpha = beta gives exactly 0
    x = synth.vector(8, 9, n)
    y = O.gesummv(m, n, 0.75, A, 0.25, A, x, L=L)
    assert _rel(y, Am @ x) < 1e-13
    negA = np.asfortranarray(-Am)
    y0 = O.gesummv(m, n, 0.75, A, 0.75, negA, x, L=L)
    assert np.all(y0 == 0.0)
    y2 = O.gesummv(m, n, 2.0, A, 0.0, negA, x, L=L)
    assert _rel(y2, 2.0 * (Am @ x)) < 1e-13
    # DGEMV is the textbook GEMV
    yd = synth.vector(8, 10, m)
    z = O.dgemv(m, n, -1.25, A, x, 0.5, yd, L=L)
    assert _rel(z, -1.25 * (Am @ x) + 0.5 * yd) < 1e-13
    # ATAX with beta
    y = O.atax(m, n, -2.0, A, x, L=L)
    assert _rel(y, -2.0 * (Am.T @ (Am @ x))) < 1e-13


def pin_vector_special(L):
    n = 4097
    w, v, u = (synth.vector(9, k, n) for k in (0, 1, 2))
    z, r = O.axpydot(n, 0.0, w, v, u, L=L)
    assert np.array_equal(z, w)
    assert abs(r - np.dot(w, u)) < 1e-13 * np.dot(np.abs(w), np.abs(u))
    z, r = O.axpydot(n, 0.3, w, v, u, L=L)
    assert _rel(z, w - 0.3 * v) < 1e-15
    assert abs(r - np.dot(w - 0.3 * v, u)) < 1e-13 * np.dot(np.abs(z), np.abs(u))
    # u := w - alpha v (formed on the host) gives r = ||z||^2 >= 0
    zz = w - 0.3 * v
    _, r2 = O.axpydot(n, 0.3, w, v, zz, L=L)
    assert r2 > 0 and abs(r2 - np.dot(zz, zz)) < 1e-13 * np.dot(zz, zz)
    assert np.all(O.waxpby(n, 1.0, w, -1.0, w, L=L) == 0.0)
    assert _rel(O.waxpby(n, 0.5, w, 2.0, v, L=L), 0.5 * w + 2.0 * v) < 1e-15
    assert _rel(O.vadd(n, w, v, u, L=L), w + v + u) < 1e-15


def pin_ieee_and_empty(L):
    # No beta = 0 shortcut: NaN in y propagates.
    m, n = 3, 4
    A = synth.matrix(10, 0, m, n)
    x = synth.vector(10, 1, n)
    y = np.array([1.0, np.nan, 2.0])
    z = O.dgemv(m, n, 1.0, A, x, 0.0, y, L=L)
    assert np.isnan(z[1]) and np.all(np.isfinite(z[[0, 2]]))
    # Padding rows (lda > m) are never read: they hold NaN here.
    Ap = synth.matrix(10, 0, m, n, lda=m + 2)
    assert np.array_equal(O.dgemv(m, n, 1.0, Ap, x, 1.0, np.zeros(m), L=L),
                          O.dgemv(m, n, 1.0, A, x, 1.0, np.zeros(m), L=L))
    # Empty sums are zero.
    q, s = O.bicgk(0, n, np.zeros((1, n), order="F"), x, np.zeros(0), L=L)
    assert q.size == 0 and np.array_equal(s, np.zeros(n))
    q, s = O.bicgk(m, 0, np.zeros((m, 0), order="F"), np.zeros(0), y[[0, 2, 0]], L=L)
    assert np.array_equal(q, np.zeros(m)) and s.size == 0
    zt = synth.vector(10, 2, n)
    xt, wt = O.dgemvt(0, n, 1.0, 2.0, np.zeros((1, n), order="F"), np.zeros(0), zt, L=L)
    assert np.array_equal(xt, zt) and wt.size == 0
    z0, r0 = O.axpydot(0, 1.0, np.zeros(0), np.zeros(0), np.zeros(0), L=L)
    assert z0.size == 0 and r0 == 0.0


def pin_dot2_bound(L):
    # Ill-conditioned dot: pairs x_j = -x_i with y_j = y_i (1 + 2^-30 c_i), so each
    # pair nearly cancels while every product rounds.  The exact value is computed
    # with rationals; Dot2 must meet |res - d| <= u|d| + gamma_n^2 |x|^T|y|
    # (Ogita, Rump and Oishi 2005, Proposition 5.5), which is far below the
    # plain sum's error on the same data.
    h = 300
    a = synth.vector(11, 0, h) * np.exp2(np.floor(40 * (synth.vector(11, 1, h) + 1) / 2))
    b = synth.vector(11, 2, h)
    c = synth.vector(11, 3, h)
    x = np.concatenate([a, -a])
    y = np.concatenate([b, b * (1.0 + 2.0 ** -30 * c)])
    perm = np.argsort(synth.vector(11, 4, 2 * h))
    x, y = x[perm], y[perm]
    exact = sum((Fraction(float(p)) * Fraction(float(q)) for p, q in zip(x, y)), Fraction(0))
    res = O.dot2(x, y, L=L)
    u = 2.0 ** -53
    n = len(x)
    gamma = n * u / (1 - n * u)
    absdot = float(np.dot(np.abs(x), np.abs(y)))
    bound = u * abs(float(exact)) + gamma ** 2 * absdot
    err = abs(Fraction(res) - exact)
    assert err <= Fraction(bound), (res, float(exact), float(err), bound)
    plain = 0.0
    for p, q in zip(x, y):
        plain += p * q
    assert abs(Fraction(plain) - exact) > 1000 * Fraction(bound)


def pin_mrhs_and_row_dot(L):
    # Multi-RHS BICGK column by column against exact int64 products, and the
    # sampled-row helper against the same exact sums.
    m, n, k = 45, 38, 5
    A = _imat(12, 0, m, n)
    Ai = A.astype(np.int64)
    P = np.asfortranarray(np.stack([_ints(12, 1 + c, n) for c in range(k)], axis=1))
    R = np.asfortranarray(np.stack([_ints(12, 10 + c, m) for c in range(k)], axis=1))
    Q, S = O.bicgk_mrhs(m, n, k, A, P, R, L=L)
    assert np.array_equal(Q, (Ai @ P.astype(np.int64)).astype(float))
    assert np.array_equal(S, (Ai.T @ R.astype(np.int64)).astype(float))
    for i in (0, 17, m - 1):
        assert O.row_dot(A[i], P[:, 0], L=L) == float(Ai[i] @ P[:, 0].astype(np.int64))


# ---------------------------------------------------------------- sparse (CSR)
def _densify(m, n, rp, col, val):
    A = np.zeros((max(m, 1), n))
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            A[i, col[k]] += val[k]
    return A[:m]


def pin_csr_golden(L):
    g, e = load("csr_bicgk_3x4.txt")
    rp, col = g["row_ptr"].astype(np.int64), g["col"].astype(np.int32)
    q, s = O.csr_bicgk(g["m"], g["n"], rp, col, g["val"], g["p"], g["r"], L=L)
    assert np.array_equal(q, e["q"]) and np.array_equal(s, e["s"])
    y = O.csr_atax(g["m"], g["n"], float(g["beta"]), rp, col, g["val"], g["p"], L=L)
    assert np.array_equal(y, e["y"])


def pin_csr_integer_exact(L):
    """Integer-valued entries and vectors: every partial sum is exact, so the
    CSR results equal exact int64 products of the densified matrix."""
    m, n = 23, 17
    rp, col, _ = synth.csr(3, 80, m, n, 5)
    val = _ints(3, 90, len(col))
    p, r = _ints(3, 91, n), _ints(3, 92, m)
    Ai = _densify(m, n, rp, col, val).astype(np.int64)
    q, s = O.csr_bicgk(m, n, rp, col, val, p, r, L=L)
    assert np.array_equal(q, (Ai @ p.astype(np.int64)).astype(float))
    assert np.array_equal(s, (Ai.T @ r.astype(np.int64)).astype(float))
    y = O.csr_atax(m, n, 2.0, rp, col, val, p, L=L)
    assert np.array_equal(y, (2 * (Ai.T @ (Ai @ p.astype(np.int64)))).astype(float))


def pin_csr_identity(L):
    n = 6
    rp, col = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32)
    p, r = np.arange(1.0, n + 1), np.arange(-3.0, n - 3)
    q, s = O.csr_bicgk(n, n, rp, col, np.ones(n), p, r, L=L)
    assert np.array_equal(q, p) and np.array_equal(s, r)


# ---------------------------------------------------------------- banded / triangular
def _g1(g, k):
    return int(np.asarray(g[k]).ravel()[0])


def pin_band_golden(L):
    g, e = load("band_bicgk_4x5.txt")
    m, n, kl, ku, ld = g["m"], g["n"], _g1(g, "kl"), _g1(g, "ku"), _g1(g, "ld")
    q, s = O.band_bicgk(BU.BAND, m, n, kl, ku, 0, g["A"], ld, g["p"], g["r"], L=L)
    assert np.array_equal(q, e["q"]) and np.array_equal(s, e["s"]), (q, s)
    y = O.band_atax(BU.BAND, m, n, kl, ku, 0, float(g["beta"]), g["A"], ld, g["p"], L=L)
    assert np.array_equal(y, e["y"]), y

    g, e = load("tri_upper_3.txt")
    n = g["n"]
    for st, A, ld in ((BU.FULL, g["full"], n), (BU.PACKED, g["packed"], 1)):
        q, s = O.band_bicgk(st, n, n, 0, n - 1, 0, A, ld, g["p"], g["r"], L=L)
        assert np.array_equal(q, e["q"]) and np.array_equal(s, e["s"]), (st, q, s)
        q, s = O.band_bicgk(st, n, n, 0, n - 1, 1, A, ld, g["p"], g["r"], L=L)
        assert np.array_equal(q, e["qu"]) and np.array_equal(s, e["su"]), (st, q, s)
        y = O.band_atax(st, n, n, 0, n - 1, 0, float(g["beta"]), A, ld, g["p"], L=L)
        assert np.array_equal(y, e["y"]), (st, y)

    g, e = load("tri_lower_unit_3.txt")
    n = g["n"]
    q, s = O.band_bicgk(BU.PACKED, n, n, n - 1, 0, 1, g["packed"], 1, g["p"], g["r"], L=L)
    assert np.array_equal(q, e["q"]) and np.array_equal(s, e["s"]), (q, s)


# (m, n, kl, ku): general bands, bands wider than the matrix, diagonal only,
# both triangles of square and rectangular matrices.
BAND_SHAPES = [(9, 7, 2, 1), (7, 11, 0, 3), (12, 5, 4, 0), (8, 8, 0, 7), (8, 8, 7, 0),
               (6, 9, 20, 20), (10, 10, 0, 0), (1, 6, 0, 5), (6, 1, 5, 0), (13, 13, 3, 3)]


def pin_band_integer_exact(L):
    """Integer-valued entries and vectors: every partial sum is exact, so the
    band results equal exact int64 products of the dense matrix, in every
    storage kind the shape allows, with and without a unit diagonal."""
    for k, (m, n, kl, ku) in enumerate(BAND_SHAPES):
        D = BU.dense(4, 100 + k, m, n, kl, ku, kind=synth.KIND_INTEGER)
        p, r = _ints(4, 120 + k, n), _ints(4, 140 + k, m)
        for unit in (0, 1):
            Du = D.copy()
            if unit:
                np.fill_diagonal(Du, 1.0)
            Di = Du.astype(np.int64)
            kinds = [BU.FULL, BU.BAND] + ([BU.PACKED] if m == n and (kl == 0 and ku == n - 1
                                                                     or ku == 0 and kl == m - 1) else [])
            for st in kinds:
                A, ld = BU.store(D, st, kl, ku)
                if unit and st != BU.PACKED:
                    # the stored diagonal must not be read: poison it
                    A = A.copy()
                    for i in range(min(m, n)):
                        A[(i + i * ld) if st == BU.FULL else (ku + i * ld)] = np.nan
                q, s = O.band_bicgk(st, m, n, kl, ku, unit, A, ld, p, r, L=L)
                assert np.array_equal(q, (Di @ p.astype(np.int64)).astype(float)), (m, n, kl, ku, st, unit)
                assert np.array_equal(s, (Di.T @ r.astype(np.int64)).astype(float)), (m, n, kl, ku, st, unit)
                y = O.band_atax(st, m, n, kl, ku, unit, -2.0, A, ld, p, L=L)
                assert np.array_equal(y, (-2 * (Di.T @ (Di @ p.astype(np.int64)))).astype(float)), (m, n, st)


def pin_band_closed_forms(L):
    n = 12
    p, r = _ints(5, 1, n), _ints(5, 2, n)
    # all-ones upper triangle: q_i = p_i + ... + p_{n-1}, s_j = r_0 + ... + r_j
    ones = np.ones(n * (n + 1) // 2)
    q, s = O.band_bicgk(BU.PACKED, n, n, 0, n - 1, 0, ones, 1, p, r, L=L)
    assert np.array_equal(q, np.cumsum(p[::-1])[::-1]) and np.array_equal(s, np.cumsum(r))
    # lower: q_i = p_0 + ... + p_i, s_j = r_j + ... + r_{n-1}
    q, s = O.band_bicgk(BU.PACKED, n, n, n - 1, 0, 0, ones, 1, p, r, L=L)
    assert np.array_equal(q, np.cumsum(p)) and np.array_equal(s, np.cumsum(r[::-1])[::-1])
    # tridiagonal (-1, 2, -1) in band storage: q = minus the second difference
    # of p; with p_i = i^2 every interior q_i is -2
    AB = np.tile(np.array([-1.0, 2.0, -1.0]), n)
    pq = np.arange(n, dtype=float) ** 2
    q, s = O.band_bicgk(BU.BAND, n, n, 1, 1, 0, AB, 3, pq, pq, L=L)
    assert np.array_equal(q[1:-1], np.full(n - 2, -2.0)) and q[0] == -1.0 and q[-1] == 2 * pq[-1] - pq[-2]
    assert np.array_equal(q, s)   # the matrix is symmetric


def pin_band_identity_and_storage(L):
    """Floating-point values: the adjoint identity r^T q = s^T p, and the
    three storage kinds of one matrix give bitwise equal results (they hold
    the same values and the definition reads them in the same order)."""
    for k, (m, n, kl, ku) in enumerate(BAND_SHAPES):
        D = BU.dense(6, 200 + k, m, n, kl, ku)
        p, r = synth.vector(6, 220 + k, n), synth.vector(6, 240 + k, m)
        A, ld = BU.store(D, BU.FULL, kl, ku)
        q, s = O.band_bicgk(BU.FULL, m, n, kl, ku, 0, A, ld, p, r, L=L)
        sc = np.abs(r) @ np.abs(D) @ np.abs(p) + 1e-300
        assert abs(r @ q - s @ p) <= 1e-13 * sc, (m, n, kl, ku)
        assert _rel(q, D @ p) < 1e-14 and _rel(s, D.T @ r) < 1e-14, (m, n, kl, ku)
        A2, ld2 = BU.store(D, BU.BAND, kl, ku)
        q2, s2 = O.band_bicgk(BU.BAND, m, n, kl, ku, 0, A2, ld2, p, r, L=L)
        assert np.array_equal(q, q2) and np.array_equal(s, s2), (m, n, kl, ku)
        if m == n and (kl == 0 and ku == n - 1 or ku == 0 and kl == m - 1):
            q3, s3 = O.band_bicgk(BU.PACKED, m, n, kl, ku, 0, BU.store_packed(D, kl == 0), 1, p, r, L=L)
            assert np.array_equal(q, q3) and np.array_equal(s, s3), (m, n, kl, ku)
    # an Inf in p meets only the band: rows whose band misses column j stay finite
    n = 8
    D = BU.dense(6, 300, n, n, 1, 1)
    A, ld = BU.store(D, BU.BAND, 1, 1)
    p = np.ones(n)
    p[5] = np.inf
    q, _ = O.band_bicgk(BU.BAND, n, n, 1, 1, 0, A, ld, p, np.ones(n), L=L)
    assert np.all(np.isfinite(q[:4])) and np.all(np.isfinite(q[7:])) and not np.isfinite(q[5])


PINS = [pin_golden, pin_integer_exact, pin_closed_forms, pin_identities,
        pin_vector_special, pin_ieee_and_empty, pin_dot2_bound, pin_mrhs_and_row_dot,
        pin_csr_golden, pin_csr_integer_exact, pin_csr_identity,
        pin_band_golden, pin_band_integer_exact, pin_band_closed_forms, pin_band_identity_and_storage]
