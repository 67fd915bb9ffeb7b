"""One runner per Table I kernel: seeded inputs, the GPU call through the C
ABI (fused or unfused form), and the oracle's result on the same inputs.
Each runner returns {output name: (gpu array, oracle array)}."""
import numpy as np

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from gpu_util import Out, dev, p, ws, sync

KINDS = {"uniform": synth.KIND_UNIFORM, "integer": synth.KIND_INTEGER}

# Form name -> (entry point name pattern, workspace form code).
FORMS = {"fused": ("bto_%s", bto.BTO_FORM_FUSED), "unfused": ("bto_unfused_%s", bto.BTO_FORM_UNFUSED),
         "df": ("bto_%s_df", bto.BTO_FORM_DF), "df_unfused": ("bto_unfused_%s_df", bto.BTO_FORM_DF_UNFUSED)}


def entry(kernel, form):
    """The entry point of `kernel` in `form` and its workspace form code."""
    name, code = FORMS[form]
    return getattr(bto, name % kernel), code


def _v(seed, aid, n, kind):
    return synth.vector(seed, aid, n, kind)


def _m(seed, aid, m, n, lda, kind):
    return synth.matrix(seed, aid, m, n, lda=lda, kind=kind)


def run_bicgk(m, n, lda, kind, seed=1, form="fused", alpha=None, beta=None):
    A = _m(seed, 0, m, n, lda, kind)
    pv, rv = _v(seed, 1, n, kind), _v(seed, 2, m, kind)
    dA, dp, dr = dev(A), dev(pv), dev(rv)
    q, s = Out(m), Out(n)
    f, code = entry("bicgk", form)
    w, nb = ws("bicgk", code, m, n)
    f(m, n, p(dA), lda, p(dp), p(dr), q.ptr(), s.ptr(), p(w), nb, None)
    sync()
    qo, so = O.bicgk(m, n, A, pv, rv)
    return {"q": (q.host(), qo), "s": (s.host(), so)}


def run_atax(m, n, lda, kind, seed=1, form="fused", alpha=None, beta=1.5):
    A = _m(seed, 0, m, n, lda, kind)
    xv = _v(seed, 1, n, kind)
    dA, dx = dev(A), dev(xv)
    y = Out(n)
    f, code = entry("atax", form)
    w, nb = ws("atax", code, m, n)
    f(m, n, beta, p(dA), lda, p(dx), y.ptr(), p(w), nb, None)
    sync()
    if form != "unfused" and m > 0 and n > 0:
        assert bto.bto_device_status(p(w)) == 0
    return {"y": (y.host(), O.atax(m, n, beta, A, xv))}


def run_gemver(m, n, lda, kind, seed=1, form="fused", alpha=1.5, beta=1.2, ldb=None):
    ldb = lda if ldb is None else ldb
    ids = synth.GEMVER_IDS
    A = _m(seed, ids["A"], m, n, lda, kind)
    u1, u2, yv = (_v(seed, ids[k], m, kind) for k in ("u1", "u2", "y"))
    v1, v2, zv = (_v(seed, ids[k], n, kind) for k in ("v1", "v2", "z"))
    dA = dev(A)
    d = [dev(a) for a in (u1, v1, u2, v2, yv, zv)]
    B = Out(ldb * n if n else 0)
    x, w_ = Out(n), Out(m)
    f, code = entry("gemver", form)
    wk, nb = ws("gemver", code, m, n)
    f(m, n, alpha, beta, p(dA), lda, *[p(t) for t in d], B.ptr(), ldb, x.ptr(), w_.ptr(), p(wk), nb, None)
    sync()
    Bo, xo, wo = O.gemver(m, n, alpha, beta, A, u1, v1, u2, v2, yv, zv)
    Bg = B.host().reshape((n, ldb)).T[:m] if n else np.zeros((m, 0))
    return {"B": (Bg, Bo), "x": (x.host(), xo), "w": (w_.host(), wo)}


def run_gesummv(m, n, lda, kind, seed=1, form="fused", alpha=1.5, beta=-0.75):
    A = _m(seed, 0, m, n, lda, kind)
    Bm = _m(seed, 1, m, n, lda, kind)
    xv = _v(seed, 2, n, kind)
    dA, dB, dx = dev(A), dev(Bm), dev(xv)
    y = Out(m)
    f, code = entry("gesummv", form)
    w, nb = ws("gesummv", code, m, n)
    f(m, n, alpha, p(dA), lda, beta, p(dB), lda, p(dx), y.ptr(), p(w), nb, None)
    sync()
    return {"y": (y.host(), O.gesummv(m, n, alpha, A, beta, Bm, xv))}


def run_dgemv(m, n, lda, kind, seed=1, form="fused", alpha=1.5, beta=-0.5):
    A = _m(seed, 0, m, n, lda, kind)
    xv, yv = _v(seed, 1, n, kind), _v(seed, 2, m, kind)
    dA, dx, dy = dev(A), dev(xv), dev(yv)
    z = Out(m)
    f, code = entry("dgemv", form)
    w, nb = ws("dgemv", code, m, n)
    f(m, n, alpha, p(dA), lda, p(dx), beta, p(dy), z.ptr(), p(w), nb, None)
    sync()
    return {"z": (z.host(), O.dgemv(m, n, alpha, A, xv, beta, yv))}


def run_dgemvt(m, n, lda, kind, seed=1, form="fused", alpha=1.5, beta=1.2):
    A = _m(seed, 0, m, n, lda, kind)
    yv, zv = _v(seed, 1, m, kind), _v(seed, 2, n, kind)
    dA, dy, dz = dev(A), dev(yv), dev(zv)
    x, w_ = Out(n), Out(m)
    f, code = entry("dgemvt", form)
    w, nb = ws("dgemvt", code, m, n)
    f(m, n, alpha, beta, p(dA), lda, p(dy), p(dz), x.ptr(), w_.ptr(), p(w), nb, None)
    sync()
    xo, wo = O.dgemvt(m, n, alpha, beta, A, yv, zv)
    return {"x": (x.host(), xo), "w": (w_.host(), wo)}


def run_axpydot(n, kind, seed=1, form="fused", alpha=0.75, compensated=False):
    wv, vv, uv = (_v(seed, k, n, kind) for k in (0, 1, 2))
    dw, dv, du = dev(wv), dev(vv), dev(uv)
    z, r = Out(n), Out(1)
    f, code = entry("axpydot", form)
    w, nb = ws("axpydot", code, 0, n)
    f(n, alpha, p(dw), p(dv), p(du), z.ptr(), r.ptr(), p(w), nb, None)
    sync()
    zo, ro = O.axpydot(n, alpha, wv, vv, uv, compensated=compensated)
    return {"z": (z.host(), zo), "r": (r.host(), np.array([ro]))}


def run_waxpby(n, kind, seed=1, form="fused", alpha=1.5, beta=-0.25):
    xv, yv = _v(seed, 0, n, kind), _v(seed, 1, n, kind)
    dx, dy = dev(xv), dev(yv)
    w = Out(n)
    f = bto.bto_waxpby if form == "fused" else bto.bto_unfused_waxpby
    f(n, alpha, p(dx), beta, p(dy), w.ptr(), None)
    sync()
    return {"w": (w.host(), O.waxpby(n, alpha, xv, beta, yv))}


def run_vadd(n, kind, seed=1, form="fused"):
    wv, yv, zv = (_v(seed, k, n, kind) for k in (0, 1, 2))
    dw, dy, dz = dev(wv), dev(yv), dev(zv)
    x = Out(n)
    f = bto.bto_vadd if form == "fused" else bto.bto_unfused_vadd
    f(n, p(dw), p(dy), p(dz), x.ptr(), None)
    sync()
    return {"x": (x.host(), O.vadd(n, wv, yv, zv))}


MATRIX_RUNNERS = {"bicgk": run_bicgk, "atax": run_atax, "gemver": run_gemver,
                  "gesummv": run_gesummv, "dgemv": run_dgemv, "dgemvt": run_dgemvt}
VECTOR_RUNNERS = {"axpydot": run_axpydot, "waxpby": run_waxpby, "vadd": run_vadd}
