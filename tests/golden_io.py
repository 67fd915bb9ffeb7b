"""Reader for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    inp, exp = {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "expect":
                exp[tok[1]] = np.array([float(t) for t in tok[2:]])
            else:
                vals = [float(t) for t in tok[1:]]
                inp[tok[0]] = vals[0] if len(vals) == 1 and tok[0] in (
                    "m", "n", "alpha", "beta") else np.array(vals)
    for k in ("m", "n"):
        if k in inp:
            inp[k] = int(inp[k])
    return inp, exp


def colmajor(flat, m, n):
    return np.asarray(flat, dtype=np.float64).reshape((n, m)).T.copy(order="F")
