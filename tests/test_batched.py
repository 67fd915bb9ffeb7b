"""GPU parity of the batched form (many uneven BICGK/GEMVER/ATAX/GESUMMV
instances, FP32 or BF16 storage, in one persistent launch): every instance
against the FP64 oracle on its stored values (normwise <= 1e-6; integer
inputs exact for BICGK), each instance bitwise equal alone and in the mix,
CUDA-graph replay equal to a plain run."""
import numpy as np
import pytest
import torch

import paper_1205_1098_gb300 as bto
import synth
from batch_util import Batch, logu_sizes
from gpu_util import relerr

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


def check_batch(b, exact=False):
    for i, spec in enumerate(b.specs):
        got, ref = b.result(i), b.reference(i)
        if spec[0] == "gemver":
            assert b.b_bound_ok(i), spec
        for k in range(len(ref) if spec[0] != "gemver" else 2):
            if exact and spec[0] == "bicgk":
                assert np.array_equal(got[k], ref[k]), (spec, k)
            else:
                assert relerr(got[k], ref[k]) <= TOL, (spec, k, relerr(got[k], ref[k]))


SPECS = [("bicgk", 1, 1, 1), ("gemver", 1, 1, 1), ("atax", 1, 1, 1), ("gesummv", 1, 1, 1),
         ("bicgk", 300, 517, 300), ("gemver", 300, 517, 301), ("atax", 517, 300, 517), ("gesummv", 299, 700, 304),
         ("bicgk", 2048, 37, 2048), ("gemver", 37, 2048, 40), ("atax", 37, 2000, 37), ("gesummv", 2000, 37, 2000),
         ("bicgk", 0, 50, 1), ("bicgk", 50, 0, 50), ("gemver", 0, 40, 1), ("gemver", 40, 0, 40),
         ("atax", 0, 30, 1), ("atax", 30, 0, 30), ("gesummv", 0, 30, 1), ("gesummv", 30, 0, 30),
         ("bicgk", 1000, 1000, 1003, "bf16"), ("gemver", 513, 255, 520, "bf16"), ("atax", 700, 900, 704, "bf16"),
         ("gesummv", 640, 800, 640, "bf16"), ("bicgk", 333, 257, 333, "bf16")]


@pytest.mark.parametrize("tile_cols", [16, 64, 128, 512])
def test_batch_mixed(tile_cols):
    b = Batch(SPECS, seed=7)
    assert b.run(tile_cols) == 0
    check_batch(b)


def test_batch_integer_bicgk_exact():
    b = Batch([("bicgk", 300, 517, 304), ("bicgk", 1000, 200, 1000), ("bicgk", 256, 300, 256, "bf16")], seed=8,
              kind=synth.KIND_INTEGER)
    assert b.run(64) == 0
    check_batch(b, exact=True)


def _copy_instance(dst, src, i):
    # Copies instance i's device inputs of batch `src` into the single-instance batch `dst`.
    start = 0
    for j, spec in enumerate(src.specs):
        cnt = _count(spec)
        if j == i:
            for t_dst, t_src in zip(dst.keep, src.keep[start:start + cnt]):
                t_dst.copy_(t_src)
            dst.host[0] = src.host[i]
            return
        start += cnt


def _count(spec):
    op = spec[0]
    return 1 + (1 if op == "gesummv" else 0) + {"bicgk": 2, "gemver": 6, "atax": 1, "gesummv": 1}[op] + \
        {"bicgk": 2, "gemver": 2, "atax": 1, "gesummv": 1}[op] + (1 if op == "gemver" else 0)


def test_batch_logu_alone_vs_mix_and_graph():
    specs = [(op, m, n, m) for (op, m, n) in logu_sizes(3, 160, 32, 1024, ops=("bicgk", "gemver", "atax", "gesummv"))]
    b = Batch(specs, seed=9)
    assert b.run(128) == 0
    check_batch(b)
    mixed = [b.result(i) for i in range(len(specs))]
    for i in (0, 17, 99, 159):
        one = Batch([specs[i]], seed=9)
        _copy_instance(one, b, i)
        assert one.run(128) == 0
        for k, (g1, g2) in enumerate(zip(one.result(0), mixed[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (specs[i], k)
    assert b.run(128, graph=True, reps=2) == 0
    for i in range(len(specs)):
        for k, (g1, g2) in enumerate(zip(b.result(i), mixed[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (specs[i], k)


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
def test_batch_submit_equals_prepare_run(pinned):
    """bto_batch_submit (counters zeroed in the uploaded plan, only non-empty
    queues launched, grids sized to their items) gives the bits of
    bto_batch_prepare + bto_batch_run, through pageable or pinned staging;
    a tiny staging buffer falls back to the pageable copy."""
    specs = [(op, m, n, m) for (op, m, n) in logu_sizes(5, 40, 32, 700, ops=("bicgk", "gemver", "atax", "gesummv"))]
    specs += [("bicgk", 300, 200, 300, "bf16"), ("atax", 257, 129, 257, "bf16")]
    b = Batch(specs, seed=11)
    assert b.run(64) == 0
    ref = [b.result(i) for i in range(len(specs))]
    for staging in ([torch.empty(1 << 20, dtype=torch.uint8, pin_memory=True),
                     torch.empty(64, dtype=torch.uint8, pin_memory=True)] if pinned else [None]):
        for out, Bout in b.outs:
            for to, _ in out:
                to.fill_(float("nan"))
            if Bout is not None:
                Bout.fill_(0)
        assert b.submit(64, staging) == 0
        for i in range(len(specs)):
            for k, (g1, g2) in enumerate(zip(b.result(i), ref[i])):
                assert np.array_equal(g1, g2, equal_nan=True), (specs[i], k)


TALL = [("bicgk", 5000, 700, 5000), ("gemver", 4500, 1300, 4500), ("atax", 4400, 520, 4400),
        ("gesummv", 4100, 600, 4104), ("bicgk", 4400, 1100, 4400, "bf16"), ("gemver", 4200, 700, 4208, "bf16"),
        ("atax", 6000, 333, 6000, "bf16"), ("gesummv", 4097, 515, 4104, "bf16"), ("bicgk", 4099, 9, 4100)]


@pytest.mark.parametrize("tile_cols", [64, 512])
def test_batch_tall_and_wide_tma(tile_cols):
    """Instances taller than one 2048-row tile and wider than one panel (several
    row-tile partials per column, several panel partials per row) on the TMA
    path, in FP32 and BF16, with ragged last tiles; equal alone and in the mix."""
    b = Batch(TALL, seed=13)
    assert b.run(tile_cols) == 0
    check_batch(b)
    mixed = [b.result(i) for i in range(len(TALL))]
    one = Batch([TALL[5]], seed=13)
    _copy_instance(one, b, 5)
    assert one.run(tile_cols) == 0
    for k, (g1, g2) in enumerate(zip(one.result(0), mixed[5])):
        assert np.array_equal(g1, g2, equal_nan=True), k


# Every instance FP32 with 16-byte leading dimensions: the whole batch is one
# cooperative launch (both stages and their combines behind grid barriers).
ONE = [("bicgk", 1000, 700, 1000), ("gemver", 1300, 900, 1300), ("atax", 800, 1200, 800),
       ("gesummv", 640, 700, 640), ("bicgk", 4400, 600, 4400), ("gemver", 2100, 1500, 2100),
       ("atax", 5000, 300, 5000), ("gemver", 4, 4, 4), ("bicgk", 4100, 9, 4100)]


@pytest.mark.parametrize("tile_cols", [64, 512])
def test_batch_one_launch_form(tile_cols):
    """The one-launch form: taken for a single-type, TMA-suited batch (and not
    once a BF16 instance joins it); every instance against the oracle; the
    bits of the multi-launch form for the same instances; graph replay and
    bto_batch_submit equal to a plain run."""
    b = Batch(ONE, seed=17)
    assert b.run(tile_cols) == 0
    assert bto.bto_batch_one_launch(b.ws)
    check_batch(b)
    ref = [b.result(i) for i in range(len(ONE))]
    mixed = Batch(ONE + [("bicgk", 300, 200, 300, "bf16")], seed=17)
    assert mixed.run(tile_cols) == 0
    assert not bto.bto_batch_one_launch(mixed.ws)
    for i in range(len(ONE)):
        for k, (g1, g2) in enumerate(zip(mixed.result(i), ref[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (ONE[i], k)
    assert b.run(tile_cols, graph=True, reps=3) == 0
    assert b.submit(tile_cols) == 0
    assert bto.bto_batch_one_launch(b.ws)
    for i in range(len(ONE)):
        for k, (g1, g2) in enumerate(zip(b.result(i), ref[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (ONE[i], k)


def test_batch_one_launch_barrier_times_out_and_context_survives():
    """A block that never arrives at the one-launch form's grid barrier: every
    wait expires into the status word (no device fault); after preparing the
    workspace again, a run succeeds with the usual results."""
    b = Batch(ONE[:4], seed=19)
    assert b.run(128) == 0 and bto.bto_batch_one_launch(b.ws)
    ref = [b.result(i) for i in range(4)]
    nb = bto.bto_batch_workspace_bytes(b.descs, 128)
    bto.bto_debug_batch_stall(b.ws, nb, 3, 50, None)
    assert bto.bto_device_status(b.ws) == bto.BTO_ERR_TIMEOUT
    assert b.run(128) == 0
    for i in range(4):
        for k, (g1, g2) in enumerate(zip(b.result(i), ref[i])):
            assert np.array_equal(g1, g2, equal_nan=True), (ONE[i], k)
