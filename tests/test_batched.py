"""GPU parity of the batched form (many uneven BICGK/GEMVER instances in one
persistent launch, FP32): every instance against the FP64 oracle on its
stored FP32 values (normwise <= 1e-6; integer inputs exact), each instance
bitwise equal alone and in the mix, CUDA-graph replay equal to a plain run."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from batch_util import Batch, logu_sizes
from gpu_util import relerr

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


def oracle_instance(b, i):
    op, m, n, lda = b.specs[i]
    A, ins = b.host[i]
    A64 = A[:m].astype(np.float64) if m else np.zeros((1, n))
    v = [x.astype(np.float64) for x in ins]
    if op == "bicgk":
        q, s = O.bicgk(m, n, A64, v[0], v[1])
        return [q, s]
    B, x, w = O.gemver(m, n, 1.5, 1.25, A64, *v)
    # x, w against the oracle run on the returned B (B is formed in FP32)
    return [x, w, B]


def check_batch(b, exact=False):
    for i, spec in enumerate(b.specs):
        got = b.result(i)
        ref = oracle_instance(b, i)
        op, m, n, lda = spec
        if op == "gemver":
            Bg = got[2]
            zm, zn = np.zeros(m), np.zeros(n)
            _, A, ins = None, *b.host[i]
            v = [x.astype(np.float64) for x in ins]
            _, xo, wo = O.gemver(m, n, 1.5, 1.25, Bg if m else np.zeros((1, n)), zm, zn, zm, zn, v[4], v[5])
            ref = [xo, wo, ref[2]]
            mag = np.abs(A[:m]).astype(np.float64) + np.abs(np.outer(v[0], v[1])) + np.abs(np.outer(v[2], v[3]))
            assert np.all(np.abs(Bg - ref[2]) <= np.spacing(np.abs(ref[2]).astype(np.float32)) + 2.0 ** -23 * mag), spec
        for k in range(2):
            if exact and op == "bicgk":
                assert np.array_equal(got[k], ref[k]), (spec, k)
            else:
                assert relerr(got[k], ref[k]) <= TOL, (spec, k, relerr(got[k], ref[k]))


SPECS = [("bicgk", 1, 1, 1), ("gemver", 1, 1, 1), ("bicgk", 300, 517, 300), ("gemver", 300, 517, 301),
         ("bicgk", 2048, 37, 2048), ("gemver", 37, 2048, 40), ("bicgk", 0, 50, 1), ("bicgk", 50, 0, 50),
         ("gemver", 0, 40, 1), ("gemver", 40, 0, 40), ("bicgk", 1000, 1000, 1003), ("gemver", 513, 255, 513)]


@pytest.mark.parametrize("tile_cols", [16, 64, 128, 256])
def test_batch_mixed(tile_cols):
    b = Batch(SPECS, seed=7)
    assert b.run(tile_cols) == 0
    check_batch(b)


def test_batch_integer_bicgk_exact():
    b = Batch([("bicgk", 300, 517, 304), ("bicgk", 1000, 200, 1000), ("gemver", 64, 64, 64)], seed=8,
              kind=synth.KIND_INTEGER)
    assert b.run(64) == 0
    check_batch(b, exact=True)


def test_batch_logu_200_alone_vs_mix_and_graph():
    specs = [(op, m, n, m) for (op, m, n) in logu_sizes(3, 200, 32, 1024)]
    b = Batch(specs, seed=9)
    assert b.run(128) == 0
    check_batch(b)
    mixed = [b.result(i) for i in range(len(specs))]
    # the same instance alone gives the same bits
    for i in (0, 17, 99, 199):
        one = Batch([specs[i]], seed=9)
        one.host[0] = b.host[i]
        # rebuild inputs identically: Batch uses per-instance array ids 1000*i, so copy device data
        for t_dst, t_src in zip(one.keep, b.keep[_offsets(b, i)[0]:_offsets(b, i)[1]]):
            if t_dst.numel() == t_src.numel():
                t_dst.copy_(t_src)
        assert one.run(128) == 0
        for k, (g1, g2) in enumerate(zip(one.result(0), mixed[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (specs[i], k)
    # graph replay reproduces the plain run
    assert b.run(128, graph=True, reps=2) == 0
    for i in range(len(specs)):
        for k, (g1, g2) in enumerate(zip(b.result(i), mixed[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (specs[i], k)


def _offsets(b, i):
    # index range of instance i's tensors in b.keep (A, inputs, outputs, B)
    start = 0
    for j, (op, m, n, lda) in enumerate(b.specs):
        cnt = 1 + (2 if op == "bicgk" else 6) + 2 + (1 if op == "gemver" else 0)
        if j == i:
            return start, start + cnt
        start += cnt
    raise IndexError
