"""Pins for the plain evaluator of the statement language (oracle/spec_eval.py).

Each pin is a function (E) -> None that raises AssertionError on failure,
where E is the evaluator module (the real one, or a mutant built by the
mutation test).  They tie it to the C oracle on the six Table I matrix
kernels (two independent implementations of the same definitions), to the
hand-worked fixtures (bit for bit) and to closed forms."""
import numpy as np

import golden_io
import oracle as O

TABLE_I = {
    "bicgk": "in: A : matrix, p r : vector\nout: q s : vector\nq = A * p\ns = A' * r",
    "batax": "in: x : vector(column), beta : scalar, A : matrix(column)\nout: y : vector(column)\n"
             "{\n  y = beta * A' * (A * x)\n}",
    "gemver": "in:  A : matrix, u1 v1 u2 v2 y z : vector, alpha beta : scalar\nout: B : matrix, x w : vector\n"
              "B = A + u1 * v1' + u2 * v2'\nx = beta * B' * y + z\nw = alpha * B * x",
    "gesummv": "in: A B : matrix, x : vector, alpha beta : scalar\nout: y : vector\n"
               "y = alpha * A * x + beta * B * x",
    "dgemv": "in: A : matrix, x y : vector, alpha beta : scalar\nout: z : vector\nz = alpha * A * x + beta * y",
    "dgemvt": "in: A : matrix, y z : vector, alpha beta : scalar\nout: x w : vector\n"
              "x = beta * A' * y + z\nw = alpha * A * x",
}


def pin_matches_c_oracle(E):
    rng = np.random.default_rng(3)
    m, n = 7, 5
    A, B = rng.uniform(-1, 1, (m, n)), rng.uniform(-1, 1, (m, n))
    v = {k: rng.uniform(-1, 1, ln) for k, ln in (("u1", m), ("v1", n), ("u2", m), ("v2", n), ("ym", m),
                                                 ("zn", n), ("xn", n), ("rm", m))}
    close = lambda a, b: np.allclose(a, b, rtol=0, atol=1e-13)
    r = E.evaluate(TABLE_I["bicgk"], {"A": A, "p": v["xn"], "r": v["rm"]})
    q, s = O.bicgk(m, n, A, v["xn"], v["rm"])
    assert close(r["q"], q) and close(r["s"], s)
    r = E.evaluate(TABLE_I["batax"], {"A": A, "x": v["xn"], "beta": 0.75})
    assert close(r["y"], O.atax(m, n, 0.75, A, v["xn"]))
    r = E.evaluate(TABLE_I["gemver"], {"A": A, "u1": v["u1"], "v1": v["v1"], "u2": v["u2"], "v2": v["v2"],
                                       "y": v["ym"], "z": v["zn"], "alpha": 1.5, "beta": 1.2})
    Bo, x, w = O.gemver(m, n, 1.5, 1.2, A, v["u1"], v["v1"], v["u2"], v["v2"], v["ym"], v["zn"])
    assert close(r["B"], Bo) and close(r["x"], x) and close(r["w"], w)
    r = E.evaluate(TABLE_I["gesummv"], {"A": A, "B": B, "x": v["xn"], "alpha": 1.5, "beta": -0.75})
    assert close(r["y"], O.gesummv(m, n, 1.5, A, -0.75, B, v["xn"]))
    r = E.evaluate(TABLE_I["dgemv"], {"A": A, "x": v["xn"], "y": v["ym"], "alpha": 1.5, "beta": -0.5})
    assert close(r["z"], O.dgemv(m, n, 1.5, A, v["xn"], -0.5, v["ym"]))
    r = E.evaluate(TABLE_I["dgemvt"], {"A": A, "y": v["ym"], "z": v["zn"], "alpha": 1.5, "beta": 1.2})
    x, w = O.dgemvt(m, n, 1.5, 1.2, A, v["ym"], v["zn"])
    assert close(r["x"], x) and close(r["w"], w)


def pin_hand_worked(E):
    for fixture, spec in (("bicgk_2x3.txt", "bicgk"), ("atax_2x3.txt", "batax"), ("gemver_2x2.txt", "gemver"),
                          ("gesummv_2x2.txt", "gesummv"), ("dgemv_2x3.txt", "dgemv"),
                          ("dgemvt_2x3.txt", "dgemvt")):
        inp, exp = golden_io.load(fixture)
        m, n = inp.pop("m"), inp.pop("n")
        vals = {k: (golden_io.colmajor(v, m, n) if k in ("A", "B") else v) for k, v in inp.items()}
        got = E.evaluate(TABLE_I[spec], vals)
        for k, e in exp.items():
            g = np.asarray(got[k])
            g = g.ravel(order="F") if g.ndim == 2 else g
            assert np.array_equal(g, e), (fixture, k)


def pin_closed_forms(E):
    """A = I gives beta x for BATAX; zero updates leave B = A and x its column
    sums for y = 1; a rank-one A = a b' gives A x = a (b . x); negation and
    subtraction cancel; a nested difference keeps its sign."""
    n = 6
    x = np.arange(1.0, n + 1)
    assert np.array_equal(E.evaluate(TABLE_I["batax"], {"A": np.eye(n), "x": x, "beta": 2.0})["y"], 2 * x)
    A = np.arange(12.0).reshape(3, 4)
    r = E.evaluate(TABLE_I["gemver"], {"A": A, "u1": np.zeros(3), "v1": np.zeros(4), "u2": np.zeros(3),
                                       "v2": np.zeros(4), "y": np.ones(3), "z": np.zeros(4), "alpha": 1.0,
                                       "beta": 1.0})
    assert np.array_equal(r["B"], A) and np.array_equal(r["x"], A.sum(axis=0))
    a, b, xx = np.array([1.0, -2.0, 3.0]), np.array([2.0, 0.5, -1.0, 4.0]), np.array([1.0, 2.0, 3.0, 4.0])
    r = E.evaluate(TABLE_I["dgemv"], {"A": np.outer(a, b), "x": xx, "y": np.zeros(3), "alpha": 1.0, "beta": 0.0})
    assert np.array_equal(r["z"], a * (b @ xx))
    prog = ("in: x y : vector\nout: z w u v : vector\nz = -x - -x\nw = x - (y - x)\nu = -x + 2 * x\n"
            "v = x - y - x")
    r = E.evaluate(prog, {"x": xx, "y": 2 * xx})
    assert np.array_equal(r["z"], np.zeros(4)) and np.array_equal(r["w"], np.zeros(4))
    assert np.array_equal(r["u"], xx)              # negation applies
    assert np.array_equal(r["v"], -2 * xx)         # (x - y) - x: subtraction is left-associative


PINS = [pin_matches_c_oracle, pin_hand_worked, pin_closed_forms]
