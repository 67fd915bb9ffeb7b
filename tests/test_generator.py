"""The sequence generator: programs in the paper's statement language (Fig. 1)
are planned into fused passes of the panel engine under the reduction rule
of Section III-C, the native runtime checks the instruction lists, and on the
GPU the generated passes reproduce the plain evaluation of the same program
(oracle/spec_eval.py, itself pinned here to the C oracle and to the
hand-worked fixtures) for the Table I kernels and for sequences beyond them."""
import numpy as np
import pytest

from oracle import spec_eval as E
from spec_pins import PINS
from paper_1205_1098_gb300 import _lib, generator as G

SPECS = {
    "bicgk": """BICGK
in: A : matrix, p r : vector
out: q s : vector
q = A * p
s = A' * r""",
    "batax": """BATAX
in: x : vector(column), beta : scalar, A : matrix(column)
out: y : vector(column)
{
  y = beta * A' * (A * x)
}""",
    "batax_row": """BATAX as printed (A row-major)
in: x : vector(column), beta : scalar, A : matrix(row)
out: y : vector(column)
{
  y = beta * A' * (A * x)
}""",
    "gemver": """GEMVER
in:  A : matrix, u1 v1 u2 v2 y z : vector, alpha beta : scalar
out: B : matrix, x w : vector
B = A + u1 * v1' + u2 * v2'
x = beta * B' * y + z
w = alpha * B * x""",
    "gemver_row": """GEMVER
in:  A : matrix(row), u1 v1 u2 v2 y z : vector, alpha beta : scalar
out: B : matrix(row), x w : vector
B = A + u1 * v1' + u2 * v2'
x = beta * B' * y + z
w = alpha * B * x""",
    "gesummv": """GESUMMV
in: A B : matrix, x : vector, alpha beta : scalar
out: y : vector
y = alpha * A * x + beta * B * x""",
    "dgemv": """DGEMV
in: A : matrix, x y : vector, alpha beta : scalar
out: z : vector
z = alpha * A * x + beta * y""",
    "dgemvt": """DGEMVT
in: A : matrix, y z : vector, alpha beta : scalar
out: x w : vector
x = beta * A' * y + z
w = alpha * A * x""",
    # Sequences beyond Table I.
    "chain": """two matrices: BICGK on A feeding a product of C
in: A C : matrix, p r : vector
out: q s v : vector
q = A * p
s = A' * r
v = C * q + 2 * s""",
    "axpy_gemv": """a vector update feeding a product, plus vector terms
in: A : matrix, x z w v : vector, alpha : scalar
out: y : vector
y = A * (x + alpha * z) - 3 * w + v""",
    "rank1_row": """one scaled rank-one term on a row-major matrix
in: A : matrix(row), u v y : vector, gamma : scalar
out: B : matrix(row), x : vector
B = A + gamma * u * v'
x = B * y""",
    "four_products": """four products of one matrix, two of a second (two passes: no mode takes two inputs)
in: A D : matrix, a b c d : vector
out: e f g h k : vector
e = A * a
f = A' * b
g = A * c
h = A' * d
k = D * (e + g) - 0.5 * D * e""",
}

MODES = {
    "bicgk": ["QS"], "batax": ["Q", "S"], "batax_row": ["S", "Q"], "gemver": ["G1", "Q"],
    "gemver_row": ["G1Q", "S"], "gesummv": ["Q2"], "dgemv": ["Q"], "dgemvt": ["S", "Q"],
    "chain": ["QS", "Q"], "axpy_gemv": ["Q"], "rank1_row": ["G1"], "four_products": ["QS", "QS", "Q", "Q"],
}


@pytest.mark.parametrize("name", sorted(MODES))
def test_plans(name):
    P = G.compile(SPECS[name])
    assert [s["mode"] for s in P.passes] == MODES[name], P.describe()


def test_second_pass_over_a_matrix_runs_reversed():
    for name in ("batax", "gemver", "dgemvt"):
        P = G.compile(SPECS[name])
        assert [s["reverse"] for s in P.passes] == [False, True], name


def test_reduction_rule_separates_a_consumer_from_its_producer():
    """Section III-C: t = A x is complete only after its loop, so A' t may not
    share that pass although both read A; independent products do."""
    dep = G.compile("in: A : matrix, x : vector\nout: y : vector\nt = A * x\ny = A' * t")
    assert [s["mode"] for s in dep.passes] == ["Q", "S"]
    ind = G.compile("in: A : matrix, x r : vector\nout: y s : vector\ny = A * x\ns = A' * r")
    assert [s["mode"] for s in ind.passes] == ["QS"]


@pytest.mark.parametrize("text,msg", [
    ("in: A : matrix, x : vector\nout: y : vector\ny = A * q", "not declared"),
    ("in: A : matrix, x : vector\nout: y : vector\nx = A * x\ny = x", "input"),
    ("in: A : matrix, x : vector\nout: y : vector\ny = A * x\ny = A' * x", "twice"),
    ("in: x z : vector\nout: y : vector\ny = x' * z", "dot products"),
    ("in: A C : matrix, x : vector\nout: y : vector\ny = A * C * x", "matrix-matrix"),
    ("in: A : matrix, u v : vector, c : scalar\nout: B : matrix\nB = c * A + u * v'", "unscaled"),
    ("in: A : tensor\nout: y : vector\ny = A", "unknown type"),
    ("in: A : matrix, x : vector\nout: y w : vector\ny = A * x", "never assigned"),
    ("in: A : matrix(row), u v : vector\nout: B : matrix\nB = A + u * v'", "storage order"),
])
def test_rejected_programs(text, msg):
    with pytest.raises(G.SpecError) as e:
        G.compile(text)
    assert msg in str(e.value)


# ------------------------------------------------------------------ oracle pins


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_spec_eval_pins(pin):
    """The plain evaluator against the C oracle, the hand-worked fixtures and
    closed forms (tests/spec_pins.py)."""
    pin(E)


# ------------------------------------------------------------------ native check (CPU)


def _shapes(P, m, n):
    """Input matrix shapes that fit every program above: A and B m x n, C and D n x m."""
    shapes = {"A": (m, n), "B": (m, n), "C": (n, m), "D": (n, m)}
    return {k: v for k, v in shapes.items() if k in P.decls and P.decls[k][2] == "in"}


def _bind(P, m, n, shapes, device="cpu"):
    import torch
    b = {}
    for k, d in P.decls.items():
        if d[0] == "scalar":
            b[k] = 1.25
        elif d[0] == "matrix":
            r, c = shapes[k] if k in shapes else shapes[P.matrix_outs[k]]
            b[k] = torch.zeros(r * c, dtype=torch.float64, device=device)
        else:
            ln = P.vector_length(k, shapes)
            b[k] = torch.zeros(max(ln, 1), dtype=torch.float64, device=device)
    return b


def test_generated_programs_pass_the_native_check(tmp_path):
    from paper_1205_1098_gb300 import build
    build.build()
    m, n = 40, 30
    for name, text in SPECS.items():
        P = G.compile(text)
        shapes = _shapes(P, m, n)
        b = _bind(P, m, n, dict(shapes))
        prog, keep = P.program(b, shapes, device="cpu")
        st, bad = _lib.bto_program_check(prog)
        assert st == _lib.BTO_OK and bad == -1, (name, bad)


def test_bound_buffers_are_checked():
    import torch
    P = G.compile(SPECS["dgemv"])
    b = _bind(P, 40, 30, {"A": (40, 30)})
    for name, bad in (("x", b["x"].float()), ("A", b["A"].view(40, 30).t()), ("alpha", "1.5")):
        bb = dict(b)
        bb[name] = bad
        with pytest.raises(G.SpecError):
            P.program(bb, {"A": (40, 30)}, device="cpu")
    with pytest.raises(G.SpecError):          # a host tensor for a device program
        P.program(b, {"A": (40, 30)}, device="cuda")
    assert P.program(b, {"A": (40, 30)}, device="cpu")[0] is not None
    assert torch.float64 == b["x"].dtype


def test_inconsistent_shapes_are_rejected():
    P = G.compile(SPECS["four_products"])
    with pytest.raises(G.SpecError):
        P.program(_bind(P, 40, 30, {"A": (40, 30), "D": (30, 40)}), {"A": (40, 30), "D": (40, 30)}, device="cpu")


def test_native_check_rejects_broken_programs():
    from paper_1205_1098_gb300 import build
    build.build()
    P = G.compile(SPECS["dgemvt"])
    b = _bind(P, 40, 30, {"A": (40, 30)})
    prog, keep = P.program(b, {"A": (40, 30)}, device="cpu")
    n = len(prog)
    # A combine that reads a slot no pass has written yet.
    bad = (_lib.Instr * n)(*prog)
    bad[1].src1 = 7
    assert _lib.bto_program_check(bad) == (_lib.BTO_ERR_INVALID_VALUE, 1)
    # A pass whose slot is written twice.
    bad = (_lib.Instr * n)(*prog)
    bad[2].slot_q = bad[0].slot_s
    assert _lib.bto_program_check(bad) == (_lib.BTO_ERR_INVALID_VALUE, 2)
    # A leading dimension shorter than the stored rows.
    bad = (_lib.Instr * n)(*prog)
    bad[0].lda = 39
    assert _lib.bto_program_check(bad) == (_lib.BTO_ERR_INVALID_VALUE, 0)
    # A combine whose length differs from its slot's.
    bad = (_lib.Instr * n)(*prog)
    bad[3].n = 31
    assert _lib.bto_program_check(bad)[1] == 3
    # An unknown instruction, and a WAXPBY writing over its input.
    bad = (_lib.Instr * n)(*prog)
    bad[1].op = 9
    assert _lib.bto_program_check(bad)[1] == 1
    w = (_lib.Instr * 1)()
    w[0].op, w[0].n, w[0].out, w[0].x, w[0].y = _lib.BTO_INSTR_WAXPBY, 4, 4096, 4096 + 16, 8192
    assert _lib.bto_program_check(w) == (_lib.BTO_ERR_INVALID_VALUE, 0)


# ------------------------------------------------------------------ GPU


def _device_inputs(P, shapes, seed, lds=None):
    """Seeded inputs: host values for the oracle, device buffers in each
    matrix's storage order (with optional padded leading dimensions)."""
    import torch
    import synth
    host, dev = {}, {}
    lds = lds or {}
    aid = 0
    for k, d in sorted(P.decls.items()):
        aid += 1
        if d[0] == "scalar":
            host[k] = dev[k] = [1.5, -0.75, 1.2, 0.5][aid % 4]
        elif d[0] == "matrix":
            if d[2] == "in":
                r, c = shapes[k]
                Av = synth.matrix(seed, aid, r, c)[:r]
                host[k] = Av
                row = P.orient[k] == "row"
                ld = lds.get(k, c if row else r)
                buf = np.full((max(r, 1), ld) if row else (max(c, 1), ld), np.nan)
                if row:
                    buf[:r, :c] = Av
                else:
                    buf[:c, :r] = Av.T
                dev[k] = torch.from_numpy(np.ascontiguousarray(buf.ravel())).cuda()
            else:
                base = P.matrix_outs[k]
                dev[k] = torch.full_like(dev[base], np.nan) if base in dev else None
        else:
            ln = P.vector_length(k, shapes)
            if d[2] == "in":
                host[k] = synth.vector(seed, 100 + aid, ln)
                dev[k] = torch.from_numpy(host[k].copy()).cuda()
            else:
                dev[k] = torch.full((max(ln, 1),), np.nan, dtype=torch.float64, device="cuda")
    return host, dev


def _check_against_oracle(P, text, shapes, seed, lds=None, tol=1e-12):
    from gpu_util import relerr
    import torch
    host, dev = _device_inputs(P, shapes, seed, lds)
    P.run(dev, shapes, lds)
    torch.cuda.synchronize()
    ref = E.evaluate(text, host)
    for k, d in P.decls.items():
        if d[2] != "out":
            continue
        if d[0] == "matrix":
            r, c = shapes.get(k, shapes[P.matrix_outs[k]])
            row = P.orient[k] == "row"
            ld = (lds or {}).get(k, (lds or {}).get(P.matrix_outs[k], c if row else r))
            g = dev[k].cpu().numpy().reshape((max(r, 1), ld) if row else (max(c, 1), ld))
            got = g[:r, :c] if row else g[:c, :r].T
        else:
            got = dev[k].cpu().numpy()[:P.vector_length(k, shapes)]
        want = np.asarray(ref[k])
        assert got.shape == want.shape, k
        assert relerr(got, want) <= tol, (k, relerr(got, want))


SHAPES_GPU = [(1500, 1300), (37, 2100), (2500, 65), (1, 1), (4099, 33), (0, 7), (7, 0)]


@pytest.mark.gpu
@pytest.mark.parametrize("name", sorted(SPECS))
@pytest.mark.parametrize("m,n", SHAPES_GPU)
def test_generated_sequences_match_oracle(name, m, n):
    from paper_1205_1098_gb300 import build
    build.build()
    text = SPECS[name]
    P = G.compile(text)
    _check_against_oracle(P, text, _shapes(P, m, n), seed=31)


@pytest.mark.gpu
def test_generated_sequences_with_padded_leading_dimensions():
    from paper_1205_1098_gb300 import build
    build.build()
    for name in ("gemver", "gemver_row", "batax_row", "gesummv"):
        text = SPECS[name]
        P = G.compile(text)
        m, n = 1201, 999
        shapes = {k: (m, n) for k in ("A", "B") if k in P.decls and P.decls[k][2] == "in"}
        row = P.orient["A"] == "row"
        lds = {k: (n if row else m) + 5 for k in P.decls if P.decls[k][0] == "matrix"}
        _check_against_oracle(P, text, shapes, seed=32, lds=lds)


@pytest.mark.gpu
def test_generated_bicgk_and_dgemv_are_the_hand_written_bits():
    """Same passes, same tile plan, same combines: the generated BICGK and DGEMV
    give the hand-written entry points' bits."""
    import torch
    import paper_1205_1098_gb300 as bto
    from paper_1205_1098_gb300 import build
    build.build()
    m, n = 3001, 2777
    P = G.compile(SPECS["bicgk"])
    host, dev = _device_inputs(P, {"A": (m, n)}, seed=33)
    P.run(dev, {"A": (m, n)})
    q, s = torch.empty(m, dtype=torch.float64, device="cuda"), torch.empty(n, dtype=torch.float64, device="cuda")
    nb = bto.bto_workspace_bytes("bicgk", 0, m, n)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    bto.bto_bicgk(m, n, dev["A"], m, dev["p"], dev["r"], q, s, ws, nb)
    torch.cuda.synchronize()
    assert torch.equal(q, dev["q"][:m]) and torch.equal(s, dev["s"][:n])
    P = G.compile(SPECS["dgemv"])
    host, dev = _device_inputs(P, {"A": (m, n)}, seed=34)
    P.run(dev, {"A": (m, n)})
    z = torch.empty(m, dtype=torch.float64, device="cuda")
    nb = bto.bto_workspace_bytes("dgemv", 0, m, n)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    bto.bto_dgemv(m, n, dev["alpha"], dev["A"], m, dev["x"], dev["beta"], dev["y"], z, ws, nb)
    torch.cuda.synchronize()
    assert torch.equal(z, dev["z"][:m])
