"""The generator's plans on random programs, without a GPU: each plan is run
by a numpy model of the instruction semantics that include/bto.h gives
bto_program_run (a pass forms the products of its stored matrix into slots,
a combine adds scaled slot sums and a scaled vector, WAXPBY forms a x + b y)
and must reproduce the plain evaluation of the program (oracle/spec_eval.py).
The plans are also checked for the reduction rule: no pass reads a vector
that is completed only after it."""
import random

import numpy as np
import pytest

from oracle import spec_eval as E
from paper_1205_1098_gb300 import generator as G


def _stored(buf, name, orient):
    M = buf[name]
    return M if orient[name] == "col" else M.T


def _set_stored(buf, name, orient, S):
    buf[name] = S if orient[name] == "col" else S.T


def execute(plan, inputs, shapes):
    """Runs plan.steps on numpy arrays; returns every named buffer."""
    buf = {k: (np.asarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else v) for k, v in inputs.items()}
    for b, a in plan.matrix_outs.items():
        buf[b] = np.full(np.shape(buf[a]) if a in buf else shapes[a], np.nan)
    slots = {}
    orient = plan.orient

    def coef(f):
        v = 1.0
        for x in f:
            v *= x if isinstance(x, float) else float(inputs[x])
        return v

    for s in plan.steps:
        if s["op"] == "pass":
            S = _stored(buf, s["A"], orient)
            mode = s["mode"]
            if mode in ("G1", "G1Q"):
                S = S + np.outer(buf[s["u1"]], buf[s["v1"]]) + np.outer(buf[s["u2"]], buf[s["v2"]])
                _set_stored(buf, s["Bout"], orient, S)
            if s["slot_q"] is not None:
                slots[s["slot_q"]] = S @ buf[s["p"]]
            if s["slot_q2"] is not None:
                slots[s["slot_q2"]] = _stored(buf, s["B"], orient) @ buf[s["p"]]
            if s["slot_s"] is not None:
                slots[s["slot_s"]] = S.T @ buf[s["r"]]
        elif s["op"] == "combine":
            n = plan.vector_length(s["out"], shapes)
            if n is None:
                n = len(buf[s["x"][1]])
            out = np.zeros(n)
            if s["src1"] is not None:
                out = out + coef(s["src1"][0]) * slots[s["src1"][1]]
            if s["src2"] is not None:
                out = out + coef(s["src2"][0]) * slots[s["src2"][1]]
            if s["x"] is not None:
                out = out + coef(s["x"][0]) * buf[s["x"][1]]
            buf[s["out"]] = out
        else:
            buf[s["out"]] = coef(s["x"][0]) * buf[s["x"][1]] + coef(s["y"][0]) * buf[s["y"][1]]
    return buf


def check_reduction_rule(plan, inputs):
    """Every vector a pass reads is an input or completed by an earlier step."""
    ready = {k for k, d in plan.decls.items() if d[2] == "in"}
    for s in plan.steps:
        if s["op"] == "pass":
            for f in ("p", "r", "u1", "v1", "u2", "v2"):
                if s.get(f) is not None:
                    assert s[f] in ready, (s, f)
            if s["Bout"] is not None:
                ready.add(s["Bout"])
        else:
            for f in ("x", "y"):
                if s.get(f) is not None:
                    assert s[f][1] in ready, (s, f)
            ready.add(s["out"])


def random_program(rng):
    """A random, well-typed program over A, B (m x n) and C (n x m), each
    stored in a random order."""
    o = {k: rng.choice(["matrix", "matrix(row)"]) for k in "ABC"}
    vec = {"m": ["ym1", "ym2"], "n": ["xn1", "xn2"]}
    mats = {"m": [("A", False), ("B", False), ("C", True)],      # products giving length m
            "n": [("A", True), ("B", True), ("C", False)]}       # products giving length n
    need = {(("A", False)): "n", ("B", False): "n", ("C", True): "n",
            ("A", True): "m", ("B", True): "m", ("C", False): "m"}
    lines, outs, formed = [], [], []
    k = 0

    def vterm(cls, depth):
        r = rng.random()
        if r < 0.45 or depth > 1:
            return rng.choice(vec[cls])
        if r < 0.8:
            M, tr = rng.choice(mats[cls])
            if formed and rng.random() < 0.5:
                M = rng.choice(formed)
                tr = cls == "n"
            arg = vterm(need[(M if M in "ABC" else "A", tr)], depth + 1)
            if "*" in arg:
                arg = "(%s)" % arg          # products associate to the left
            elif rng.random() < 0.3:
                arg = "(%s + %s)" % (arg, rng.choice(vec[need[(M if M in "ABC" else "A", tr)]]))
            return "%s%s * %s" % (M, "'" if tr else "", arg)
        return "%s * %s" % (rng.choice(["2", "a", "-0.5", "b"]), rng.choice(vec[cls]))

    for _ in range(rng.randint(2, 5)):
        if rng.random() < 0.2 and not formed:
            k += 1
            name = "D%d" % k
            terms = " + ".join("%s * %s'" % (rng.choice(vec["m"]), rng.choice(vec["n"]))
                               for _ in range(rng.randint(1, 2)))
            if rng.random() < 0.3:
                terms = "a * " + terms
            lines.append("%s = A + %s" % (name, terms))
            formed.append(name)
            outs.append((name, "matrix" if o["A"] == "matrix" else "matrix(row)"))
            continue
        cls = rng.choice("mn")
        k += 1
        name = "v%s%d" % (cls, k)
        expr = " + ".join(vterm(cls, 0) for _ in range(rng.randint(1, 3)))
        if rng.random() < 0.25:
            # Two equally shaped matrices on one input (a pass of mode Q2 when
            # both are stored so that the product is the row accumulators).
            tr = "'" if cls == "n" else ""
            v = rng.choice(vec["m" if cls == "n" else "n"])
            expr = "%s * A%s * %s + B%s * %s" % (rng.choice(["a", "2"]), tr, v, tr, v)
        lines.append("%s = %s" % (name, expr))
        vec[cls].append(name)
        outs.append((name, "vector"))
    decl_in = "in: A : %s, B : %s, C : %s, ym1 ym2 xn1 xn2 : vector, a b : scalar" % (o["A"], o["B"], o["C"])
    decl_out = "out: " + ", ".join("%s : %s" % (n, t) for n, t in outs)
    return "\n".join(["random program", decl_in, decl_out] + lines)


@pytest.mark.parametrize("seed", range(60))
def test_random_programs_plan_to_the_definition(seed):
    rng = random.Random(seed)
    text = random_program(rng)
    P = G.compile(text)
    m, n = 7 + seed % 5, 4 + seed % 3
    nrng = np.random.default_rng(seed)
    inputs = {"A": nrng.uniform(-1, 1, (m, n)), "B": nrng.uniform(-1, 1, (m, n)),
              "C": nrng.uniform(-1, 1, (n, m)), "ym1": nrng.uniform(-1, 1, m), "ym2": nrng.uniform(-1, 1, m),
              "xn1": nrng.uniform(-1, 1, n), "xn2": nrng.uniform(-1, 1, n), "a": 1.5, "b": -0.75}
    shapes = {"A": (m, n), "B": (m, n), "C": (n, m)}
    check_reduction_rule(P, inputs)
    got = execute(P, inputs, shapes)
    want = E.evaluate(text, inputs)
    for k, d in P.decls.items():
        if d[2] == "out":
            assert np.allclose(got[k], want[k], rtol=1e-12, atol=1e-12), (text, P.describe(), k)


def test_model_reproduces_the_table_i_plans():
    """The model against the evaluator on the Table I programs (both storage
    orders), whose plans the GPU tests check on the runtime itself."""
    import test_generator as T
    m, n = 9, 6
    rng = np.random.default_rng(1)
    for name in ("bicgk", "batax", "batax_row", "gemver", "gemver_row", "gesummv", "dgemv", "dgemvt"):
        text = T.SPECS[name]
        P = G.compile(text)
        inputs = {}
        for k, d in P.decls.items():
            if d[2] != "in":
                continue
            if d[0] == "scalar":
                inputs[k] = 1.25
            elif d[0] == "matrix":
                inputs[k] = rng.uniform(-1, 1, (m, n))
            else:
                inputs[k] = rng.uniform(-1, 1, P.vector_length(k, {"A": (m, n)}))
        shapes = {k: (m, n) for k, d in P.decls.items() if d[0] == "matrix" and d[2] == "in"}
        got = execute(P, inputs, shapes)
        want = E.evaluate(text, inputs)
        for k, d in P.decls.items():
            if d[2] == "out":
                assert np.allclose(got[k], want[k], rtol=1e-12, atol=1e-12), (name, k)


@pytest.mark.parametrize("seed", range(0, 60, 3))
def test_every_fusion_choice_plans_to_the_definition(seed):
    """Each distinct plan the fusion policies give (the legal points a
    measured search chooses among) computes the program; Max-Fuse comes
    first and makes the fewest passes."""
    rng = random.Random(seed)
    text = random_program(rng)
    m, n = 8, 5
    nrng = np.random.default_rng(seed)
    inputs = {"A": nrng.uniform(-1, 1, (m, n)), "B": nrng.uniform(-1, 1, (m, n)),
              "C": nrng.uniform(-1, 1, (n, m)), "ym1": nrng.uniform(-1, 1, m), "ym2": nrng.uniform(-1, 1, m),
              "xn1": nrng.uniform(-1, 1, n), "xn2": nrng.uniform(-1, 1, n), "a": 1.5, "b": -0.75}
    shapes = {"A": (m, n), "B": (m, n), "C": (n, m)}
    want = E.evaluate(text, inputs)
    choices = G.fusion_choices(text)
    assert choices[0][0] == G.MAX_FUSE
    npass = [len(P.passes) for _, P in choices]
    assert npass[0] == min(npass)
    for pol, P in choices:
        check_reduction_rule(P, inputs)
        got = execute(P, inputs, shapes)
        for k, d in P.decls.items():
            if d[2] == "out":
                assert np.allclose(got[k], want[k], rtol=1e-12, atol=1e-12), (pol, k)


def test_fusion_choices_of_table_i():
    import test_generator as T
    modes = lambda name: [[s["mode"] for s in P.passes] for _, P in G.fusion_choices(T.SPECS[name])]
    assert modes("bicgk") == [["QS"], ["S", "Q"]]
    assert modes("gesummv") == [["Q2"], ["Q", "Q"]]
    assert modes("gemver") == [["G1", "Q"], ["G1", "S", "Q"]]
    assert modes("dgemv") == [["Q"]]


@pytest.mark.parametrize("orient", ["matrix", "matrix(row)"])
def test_chained_updates(orient):
    """A formed matrix updated again: each update shares its pass with a
    product of the matrix it forms (G1 or G1Q by storage order), and the
    second pass reads the first one's output."""
    text = ("chained updates\nin: A : %s, u w y : vector, v z : vector\nout: B : %s, C : %s, x s : vector\n"
            "B = A + u * v'\nC = B + w * z' + 2 * u * z'\nx = C * z\ns = B' * y" % (orient, orient, orient))
    P = G.compile(text)
    modes = [p["mode"] for p in P.passes]
    assert modes == (["G1", "G1Q"] if orient == "matrix" else ["G1Q", "G1"])
    assert P.passes[1]["A"] == "B" and P.passes[1]["Bout"] == "C" and P.passes[1]["reverse"]
    m, n = 6, 4
    rng = np.random.default_rng(0)
    inp = {"A": rng.uniform(-1, 1, (m, n)), "u": rng.uniform(-1, 1, m), "w": rng.uniform(-1, 1, m),
           "y": rng.uniform(-1, 1, m), "v": rng.uniform(-1, 1, n), "z": rng.uniform(-1, 1, n)}
    check_reduction_rule(P, inp)
    got, want = execute(P, inp, {"A": (m, n)}), E.evaluate(text, inp)
    for k in ("B", "C", "x", "s"):
        assert np.allclose(got[k], want[k], rtol=1e-12, atol=1e-12), k
