"""The all-core oracle (oracle/bto_oracle_par.c, OpenMP over independent
outputs) gives bit-identical results to the serial oracle for every Table I
sequence, on shapes with padded leading dimensions, single rows and columns,
and empty sizes (no GPU).  The benchmark's CPU baseline and reference arm time
it, so what they time is the oracle's own arithmetic."""
import numpy as np
import pytest

import oracle as O
import synth

SHAPES = [(1, 1, 1), (3, 5, 4), (257, 131, 260), (64, 1000, 64), (1000, 64, 1003), (0, 7, 1), (7, 0, 7)]


def _both(fn, *args):
    return fn(*args, L=O.lib()), fn(*args, L=O.lib_par())


def _same(a, b):
    a = a if isinstance(a, tuple) else (a,)
    b = b if isinstance(b, tuple) else (b,)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y)), "not bit-identical"


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "%dx%d_ld%d" % s)
def test_matrix_sequences_bit_identical(shape):
    m, n, lda = shape
    A = synth.matrix(5, 0, m, n, lda=lda, pad=0.0)
    B = synth.matrix(5, 1, m, n, lda=lda, pad=0.0)
    vm = [synth.vector(5, 10 + k, m) for k in range(4)]
    vn = [synth.vector(5, 20 + k, n) for k in range(4)]
    _same(*_both(O.bicgk, m, n, A, vn[0], vm[0]))
    _same(*_both(O.atax, m, n, 1.25, A, vn[0]))
    _same(*_both(O.gemver, m, n, 1.5, 1.2, A, vm[0], vn[0], vm[1], vn[1], vm[2], vn[2]))
    _same(*_both(O.gesummv, m, n, 1.5, A, -0.75, B, vn[0]))
    _same(*_both(O.dgemv, m, n, 1.5, A, vn[0], -0.5, vm[0]))
    _same(*_both(O.dgemvt, m, n, 1.5, 1.2, A, vm[0], vn[0]))


@pytest.mark.parametrize("n", [0, 1, 1000, 100003])
def test_vector_sequences_bit_identical(n):
    w, v, u = (synth.vector(6, k, n) for k in range(3))
    _same(*_both(O.axpydot, n, 0.75, w, v, u))
    _same(*_both(O.waxpby, n, 1.5, w, -0.25, v))
    _same(*_both(O.vadd, n, w, v, u))


def test_integer_inputs_exact_on_both():
    m, n = 300, 517
    A = synth.matrix(4, 0, m, n, kind=synth.KIND_INTEGER)
    p, r = synth.vector(4, 1, n, kind=synth.KIND_INTEGER), synth.vector(4, 2, m, kind=synth.KIND_INTEGER)
    (q1, s1), (q2, s2) = _both(O.bicgk, m, n, A, p, r)
    Ai = A[:m].astype(np.int64)
    assert np.array_equal(q2, Ai @ p.astype(np.int64)) and np.array_equal(s2, Ai.T @ r.astype(np.int64))
    assert np.array_equal(q1, q2) and np.array_equal(s1, s2)
