"""Storage order and transposition (the bto_*_layout entry points): on
row-major storage every FP64 sequence matches the oracle on the same
mathematical matrix; column-major calls through the layout entry points give
the ordinary entry points' bits; DGEMV with a transposition flag matches the
oracle's DGEMV of A^T; GEMVER's B is the same bits in both orders (each
element is the same two fused multiply-adds).  Argument validation runs
without a GPU."""
import numpy as np
import pytest

import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import _lib, build

ROW, COL = _lib.BTO_ROW_MAJOR, _lib.BTO_COL_MAJOR

# (m, n, lda padding): ragged shapes spanning several panels and row chunks,
# thin and flat ones, single elements and empties.
SHAPES = [(1500, 1300, 0), (1500, 1300, 3), (37, 2100, 0), (2500, 65, 1), (1, 1, 0),
          (4099, 33, 0), (0, 5, 0), (5, 0, 0)]


@pytest.fixture(scope="module")
def L():
    build.build()
    return bto.lib()


def test_layout_validation_without_gpu(L):
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_layout(2, 8, 4, 4096, 8, 4096, 8192, 12288, 16384, 0, 0, 0)
    assert e.value.status == _lib.BTO_ERR_INVALID_VALUE and e.value.arg == 1
    # Row-major: lda must cover n (arg 5), not m.
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_layout(ROW, 8, 4, 4096, 3, 4096, 8192, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 5
    # Column-major delegates; the position counts the layout argument.
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_layout(COL, 8, 4, 4096, 7, 4096, 8192, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 5
    with pytest.raises(bto.BtoError) as e:
        bto.bto_dgemv_layout(ROW, 2, 8, 4, 1.0, 4096, 4, 8192, 0.0, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 2
    with pytest.raises(bto.BtoError) as e:   # transposed: x has m elements, NULL x rejected
        bto.bto_dgemv_layout(ROW, _lib.BTO_TRANS, 8, 4, 1.0, 4096, 4, 0, 0.0, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 8
    with pytest.raises(bto.BtoError) as e:   # column-major, no transposition: bto_dgemv's lda (arg 5) + 2
        bto.bto_dgemv_layout(COL, 0, 8, 4, 1.0, 4096, 7, 8192, 0.0, 12288, 16384, 0, 0, 0)
    assert e.value.arg == 7
    with pytest.raises(bto.BtoError) as e:   # GEMVER row-major: ldb < n
        bto.bto_gemver_layout(ROW, 8, 4, 1.0, 1.0, 0x10000, 4, 64, 128, 192, 256, 320, 384, 0x20000, 3,
                              512, 576, 0, 0, 0)
    assert e.value.arg == 15
    with pytest.raises(bto.BtoError) as e:   # GESUMMV row-major: y overlaps B
        bto.bto_gesummv_layout(ROW, 8, 4, 1.0, 0x10000, 4, 1.0, 0x20000, 4, 0x30000, 0x20008, 0, 0, 0)
    assert e.value.arg == 11
    with pytest.raises(bto.BtoError) as e:
        bto.bto_layout_workspace_bytes("bicgk", ROW, _lib.BTO_TRANS, 8, 8)
    assert e.value.arg == 3
    with pytest.raises(bto.BtoError) as e:
        bto.bto_layout_workspace_bytes("axpydot", ROW, 0, 8, 8)
    assert e.value.arg == 1
    with pytest.raises(bto.BtoError) as e:
        bto.bto_layout_workspace_bytes("gemver", 5, 0, 8, 8)
    assert e.value.arg == 2


# ------------------------------------------------------------------ GPU


def _row_major(A, m, n, pad):
    """Row-major device copy of the m x n matrix A with lda = n + pad (NaN padding)."""
    import torch
    lda = max(1, n + pad)
    buf = np.full((max(m, 1), lda), np.nan)
    buf[:m, :n] = A[:m, :n]
    return torch.from_numpy(np.ascontiguousarray(buf.ravel())).cuda(), lda


def _inputs(m, n, seed=21):
    import synth
    A = synth.matrix(seed, 0, m, n)[:m]
    B = synth.matrix(seed, 1, m, n)[:m]
    v = {k: synth.vector(seed, 10 + i, ln) for i, (k, ln) in
         enumerate((("u1", m), ("v1", n), ("u2", m), ("v2", n), ("y", m), ("z", n), ("xm", m), ("xn", n)))}
    return A, B, v


def _ws(op, layout, trans, m, n):
    import torch
    nb = bto.bto_layout_workspace_bytes(op, layout, trans, m, n)
    t = torch.empty(max(nb, 1) + 256, dtype=torch.uint8, device="cuda")
    t.fill_(0xA5)
    return t, nb


def _check(got, ref, what):
    from gpu_util import TOL64, relerr
    assert got.shape == np.asarray(ref).shape, what
    assert relerr(got, ref) <= TOL64, (what, relerr(got, ref))


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,pad", SHAPES)
def test_row_major_matches_oracle(L, m, n, pad):
    import oracle as O
    from gpu_util import Out, dev, p, sync
    A, B, v = _inputs(m, n)
    dA, lda = _row_major(A, m, n, pad)
    dB, ldb = _row_major(B, m, n, pad)
    d = {k: dev(x) for k, x in v.items()}

    # BICGK
    q, s = Out(m), Out(n)
    ws, nb = _ws("bicgk", ROW, 0, m, n)
    bto.bto_bicgk_layout(ROW, m, n, dA, lda, p(d["xn"]), p(d["xm"]), q.ptr(), s.ptr(), ws, nb)
    sync()
    rq, rs = O.bicgk(m, n, A, v["xn"], v["xm"])
    _check(q.host(), rq, "bicgk q"); _check(s.host(), rs, "bicgk s")

    # BATAX
    y = Out(n)
    ws, nb = _ws("atax", ROW, 0, m, n)
    bto.bto_atax_layout(ROW, m, n, 1.25, dA, lda, p(d["xn"]), y.ptr(), ws, nb)
    sync()
    _check(y.host(), O.atax(m, n, 1.25, A, v["xn"]), "atax y")

    # GESUMMV
    y = Out(m)
    ws, nb = _ws("gesummv", ROW, 0, m, n)
    bto.bto_gesummv_layout(ROW, m, n, 1.5, dA, lda, -0.75, dB, ldb, p(d["xn"]), y.ptr(), ws, nb)
    sync()
    _check(y.host(), O.gesummv(m, n, 1.5, A, -0.75, B, v["xn"]), "gesummv y")

    # DGEMVT
    x, w = Out(n), Out(m)
    ws, nb = _ws("dgemvt", ROW, 0, m, n)
    bto.bto_dgemvt_layout(ROW, m, n, 1.5, 1.2, dA, lda, p(d["y"]), p(d["z"]), x.ptr(), w.ptr(), ws, nb)
    sync()
    rx, rw = O.dgemvt(m, n, 1.5, 1.2, A, v["y"], v["z"])
    _check(x.host(), rx, "dgemvt x"); _check(w.host(), rw, "dgemvt w")

    # GEMVER (B out of place)
    import torch
    dBo = torch.full_like(dA, np.nan)
    x, w = Out(n), Out(m)
    ws, nb = _ws("gemver", ROW, 0, m, n)
    bto.bto_gemver_layout(ROW, m, n, 1.5, 1.2, dA, lda, p(d["u1"]), p(d["v1"]), p(d["u2"]), p(d["v2"]),
                          p(d["y"]), p(d["z"]), dBo, lda, x.ptr(), w.ptr(), ws, nb)
    sync()
    rB, rx, rw = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"])
    gB = dBo.cpu().numpy().reshape(max(m, 1), lda)[:m, :n]
    _check(gB.ravel(), np.asarray(rB)[:m, :n].ravel(), "gemver B")
    _check(x.host(), rx, "gemver x"); _check(w.host(), rw, "gemver w")
    if m and n:
        # The padding columns of the row-major B are not written.
        assert np.all(np.isnan(dBo.cpu().numpy().reshape(max(m, 1), lda)[:m, n:]))


@pytest.mark.gpu
@pytest.mark.parametrize("m,n,pad", SHAPES)
@pytest.mark.parametrize("layout", [COL, ROW])
@pytest.mark.parametrize("trans", [0, 1])
def test_dgemv_transposition(L, m, n, pad, layout, trans):
    import oracle as O
    from gpu_util import Out, dev, p, sync
    A, _, v = _inputs(m, n, seed=22)
    if layout == ROW:
        dA, lda = _row_major(A, m, n, pad)
    else:
        import synth
        Af = synth.matrix(22, 0, m, n, lda=max(1, m + pad))
        dA, lda = dev(Af), max(1, m + pad)
    lx, lz = (m, n) if trans else (n, m)
    x = v["xm"] if trans else v["xn"]
    yv = v["z"] if trans else v["y"]          # length lz
    z = Out(lz)
    ws, nb = _ws("dgemv", layout, trans, m, n)
    dx, dy = dev(x), dev(yv)   # kept alive until the call has run
    bto.bto_dgemv_layout(layout, trans, m, n, 1.5, dA, lda, p(dx), -0.5, p(dy), z.ptr(), ws, nb)
    sync()
    opA = A.T if trans else A
    ref = O.dgemv(lz, lx, 1.5, np.asfortranarray(opA), x, -0.5, yv)
    _check(z.host(), ref, "dgemv z")


@pytest.mark.gpu
def test_dgemv_layout_in_place(L):
    """z == y: z <- alpha op(A) x + beta z."""
    import oracle as O
    from gpu_util import dev, sync
    m, n = 700, 1900
    A, _, v = _inputs(m, n, seed=23)
    dA, lda = _row_major(A, m, n, 0)
    zy = dev(v["z"])
    ws, nb = _ws("dgemv", ROW, 1, m, n)
    bto.bto_dgemv_layout(ROW, 1, m, n, 2.0, dA, lda, dev(v["xm"]), 0.25, zy, zy, ws, nb)
    sync()
    _check(zy.cpu().numpy(), O.dgemv(n, m, 2.0, np.asfortranarray(A.T), v["xm"], 0.25, v["z"]), "z")


@pytest.mark.gpu
def test_col_major_layout_calls_are_the_ordinary_entry_points(L):
    import torch
    from gpu_util import dev, sync
    m, n = 1300, 1100
    A, B, v = _inputs(m, n, seed=24)
    dA, dB = dev(np.asfortranarray(A)), dev(np.asfortranarray(B))
    d = {k: dev(x) for k, x in v.items()}
    outs = lambda: [torch.full((max(m, n),), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    for op in ("bicgk", "atax", "gemver", "gesummv", "dgemv", "dgemvt"):
        nb = bto.bto_workspace_bytes(op, 0, m, n)
        assert bto.bto_layout_workspace_bytes(op, COL, 0, m, n) == nb
        ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        res = []
        for via_layout in (False, True):
            o = outs()
            Bo = torch.empty(m * n, dtype=torch.float64, device="cuda")
            f = getattr(bto, "bto_" + op + ("_layout" if via_layout else ""))
            pre = (COL,) if via_layout else ()
            if op == "bicgk":
                f(*pre, m, n, dA, m, d["xn"], d["xm"], o[0], o[1], ws, nb)
            elif op == "atax":
                f(*pre, m, n, 1.25, dA, m, d["xn"], o[0], ws, nb)
            elif op == "gemver":
                f(*pre, m, n, 1.5, 1.2, dA, m, d["u1"], d["v1"], d["u2"], d["v2"], d["y"], d["z"], Bo, m,
                  o[0], o[1], ws, nb)
            elif op == "gesummv":
                f(*pre, m, n, 1.5, dA, m, -0.75, dB, m, d["xn"], o[0], ws, nb)
            elif op == "dgemv":
                if via_layout:
                    f(COL, 0, m, n, 1.5, dA, m, d["xn"], -0.5, d["y"], o[0], ws, nb)
                else:
                    f(m, n, 1.5, dA, m, d["xn"], -0.5, d["y"], o[0], ws, nb)
            else:
                f(*pre, m, n, 1.5, 1.2, dA, m, d["y"], d["z"], o[0], o[1], ws, nb)
            sync()
            res.append([t.cpu().numpy() for t in o] + ([Bo.cpu().numpy()] if op == "gemver" else []))
        for a, b in zip(*res):
            assert np.array_equal(a, b, equal_nan=True), op


@pytest.mark.gpu
def test_gemver_b_same_bits_in_both_orders_and_in_place(L):
    """Row-major B equals the column-major B bit for bit (the same two fused
    multiply-adds per element), also when B overwrites A."""
    import torch
    import oracle as O
    from gpu_util import dev, sync
    m, n = 2100, 1700
    A, _, v = _inputs(m, n, seed=25)
    d = {k: dev(x) for k, x in v.items()}
    # Column-major reference run.
    dAc = dev(np.asfortranarray(A))
    Bc = torch.empty(m * n, dtype=torch.float64, device="cuda")
    xc, wc = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (n, m))
    nb = bto.bto_workspace_bytes("gemver", 0, m, n)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    bto.bto_gemver(m, n, 1.5, 1.2, dAc, m, d["u1"], d["v1"], d["u2"], d["v2"], d["y"], d["z"], Bc, m, xc, wc,
                   ws, nb)
    # Row-major, B written over A.
    dAr, lda = _row_major(A, m, n, 0)
    xr, wr = (torch.empty(k, dtype=torch.float64, device="cuda") for k in (n, m))
    ws2, nb2 = _ws("gemver", ROW, 0, m, n)
    bto.bto_gemver_layout(ROW, m, n, 1.5, 1.2, dAr, lda, d["u1"], d["v1"], d["u2"], d["v2"], d["y"], d["z"],
                          dAr, lda, xr, wr, ws2, nb2)
    sync()
    Bcol = Bc.cpu().numpy().reshape(n, m).T
    Brow = dAr.cpu().numpy().reshape(m, lda)[:, :n]
    assert np.array_equal(Bcol, Brow)
    rB, rx, rw = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["y"], v["z"])
    _check(xr.cpu().numpy(), rx, "x"); _check(wr.cpu().numpy(), rw, "w")
