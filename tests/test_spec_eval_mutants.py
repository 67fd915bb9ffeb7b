"""Planted mistakes in the statement-language evaluator must fail a pin (no
GPU): each mutant is a copy of oracle/spec_eval.py with one plausible mistake,
loaded as its own module and run through tests/spec_pins.py."""
import importlib.util
import os

import pytest

from spec_pins import PINS

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "spec_eval.py")

MUTANTS = [
    ("transpose_ignored", "return a.T if isinstance(a, np.ndarray) else a", "return a"),
    ("minus_as_plus", "    if op == \"-\":\n        return a - b", "    if op == \"-\":\n        return a + b"),
    ("negation_dropped", "    if op == \"neg\":\n        return -a", "    if op == \"neg\":\n        return a"),
    ("plus_binds_tighter", '_PREC = {"+": 1, "-": 1, "*": 2, "neg": 3}', '_PREC = {"+": 2, "-": 1, "*": 2, "neg": 3}'),
    ("elementwise_product", "return a @ b", "return a * b.T if a.shape != b.shape else a * b"),
    ("right_associative_minus", "_PREC[stack[-1]] >= _PREC[op]", "_PREC[stack[-1]] > _PREC[op]"),
]


def _load(path, name):
    spec = importlib.util.spec_from_file_location(name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _fails(E):
    for pin in PINS:
        try:
            pin(E)
        except Exception:          # a wrong value, or an expression the mutant cannot evaluate
            return True
    return False


def test_real_evaluator_passes():
    assert not _fails(_load(SRC, "spec_eval_real"))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site must be unique: " + name
    path = tmp_path / ("spec_eval_%s.py" % name)
    path.write_text(src.replace(old, new))
    assert _fails(_load(str(path), "spec_eval_" + name)), "planted mistake %s passed every pin" % name
