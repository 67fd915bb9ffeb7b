"""Build the oracle shared library (plain C, gcc).  Test infrastructure only."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bto_oracle.c")
SRC_PAR = os.path.join(HERE, "bto_oracle_par.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
LIB_PAR = os.path.join(OUT_DIR, "liboracle_par.so")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(src=SRC, out=LIB, force=False, extra=()):
    """Compile `src` into the shared library `out` (skipped when up to date)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + list(extra) + ["-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build_par(force=False):
    """The same sequences divided over host cores (OpenMP); bit-equal results."""
    return build(SRC_PAR, LIB_PAR, force=force, extra=("-fopenmp",))


def build_all(force=False):
    return build(force=force), build_par(force=force)


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))
