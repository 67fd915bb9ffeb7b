"""The oracle and the CUDA path share no code: nothing under the package
imports, loads or names the oracle, the oracle imports nothing of the
package, and the two sides' native sources include nothing of each other.
Only the shared input generators (`synth`) may be used by both, and they
hold none of the sequences' arithmetic."""
import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1205_1098_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def _imports(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            out.add(node.module.split(".")[0])
    return out


def test_product_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _imports(f), f
        src = open(f).read()
        assert "bto_oracle" not in src and "liboracle" not in src, f


def test_oracle_never_imports_the_product():
    for f in _files(ORACLE, (".py",)):
        assert "paper_1205_1098_gb300" not in _imports(f), f


def test_native_sources_are_separate():
    for f in _files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".h")):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(f).read()):
            assert "oracle" not in inc, (f, inc)
    for f in _files(ORACLE, (".c", ".h")):
        for inc in re.findall(r'#include\s+"([^"]+)"', open(f).read()):
            assert "bto.h" not in inc and "csrc" not in inc, (f, inc)


def test_synth_holds_no_sequence_arithmetic():
    """The shared generators only map (seed, id, index) to numbers: they import
    neither side and call no product or oracle routine."""
    for f in _files(os.path.join(ROOT, "synth"), (".py",)):
        imps = _imports(f)
        assert not imps & {"oracle", "paper_1205_1098_gb300", "torch"}, (f, imps)
