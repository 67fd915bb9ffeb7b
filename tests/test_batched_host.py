"""The batched form's host side, without a GPU: bto_batch_workspace_bytes
validates every descriptor (op, storage type, sizes, leading dimensions,
operands each op needs) and the panel width before anything touches a
device, and sizes the workspace of valid batches.  Descriptors carry
made-up aligned addresses; nothing is dereferenced on the host.  The
sweep's assignment of work items to blocks (longest processing time first)
is checked through bto_debug_lpt: a hand-worked example, equal items, and
Graham's list-scheduling bound on uneven lists."""
import numpy as np
import pytest

import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import _lib, build

OP = {"bicgk": 0, "atax": 1, "gemver": 2, "gesummv": 3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _desc(d, op, m, n, lda=None, a_type=1, k=0):
    base = 0x10000000 * (k + 1)
    d.op, d.a_type, d.m, d.n = OP[op], a_type, m, n
    d.lda = d.ldb = max(1, m) if lda is None else lda
    d.alpha, d.beta = 1.5, 1.25
    d.A, d.B = base, base + 0x4000000
    for j in range(6):
        d.in_[j] = base + 0x8000000 + j * 0x100000
    for j in range(2):
        d.out[j] = base + 0xC000000 + j * 0x100000


def _batch(specs):
    descs = (bto.BatchDesc * len(specs))()
    for k, s in enumerate(specs):
        _desc(descs[k], *s, k=k)
    return descs


def test_valid_batches_are_sized():
    one = bto.bto_batch_workspace_bytes(_batch([("bicgk", 300, 200)]))
    mix = bto.bto_batch_workspace_bytes(_batch([("bicgk", 300, 200), ("gemver", 500, 700), ("atax", 64, 1000),
                                                ("gesummv", 1000, 64, None, 2)]))
    assert 0 < one < mix
    assert bto.bto_batch_workspace_bytes(_batch([])) >= 0
    # Empty instances are valid and need no operands.
    e = _batch([("gemver", 0, 5), ("bicgk", 7, 0)])
    for d in e:
        d.A = d.B = None
    assert bto.bto_batch_workspace_bytes(e) >= 0


@pytest.mark.parametrize("break_it", [
    lambda d: setattr(d, "op", 5),                  # DGEMV is not a batched op
    lambda d: setattr(d, "a_type", 0),              # FP64 storage is not a batched type
    lambda d: setattr(d, "m", -1),
    lambda d: setattr(d, "lda", 299),               # lda < m
    lambda d: setattr(d, "A", None),
    lambda d: setattr(d, "A", 0x10000002),          # not aligned to the element size
    lambda d: d.in_.__setitem__(5, None),           # GEMVER's z
    lambda d: d.out.__setitem__(1, None),           # GEMVER's w
    lambda d: setattr(d, "B", None),                # GEMVER's output matrix
    lambda d: setattr(d, "ldb", 10),
    lambda d: setattr(d, "n", 1 << 31),             # beyond int32
])
def test_invalid_descriptors_are_rejected(break_it):
    descs = _batch([("bicgk", 100, 100), ("gemver", 300, 200), ("atax", 50, 60)])
    break_it(descs[1])
    with pytest.raises(bto.BtoError) as e:
        bto.bto_batch_workspace_bytes(descs)
    assert e.value.status == _lib.BTO_ERR_INVALID_VALUE and e.value.arg == 2


def test_operands_each_op_needs():
    # ATAX reads one input and writes one output; the unused slots may be NULL.
    d = _batch([("atax", 40, 30)])
    for j in range(1, 6):
        d[0].in_[j] = None
    d[0].out[1] = None
    d[0].B = None
    assert bto.bto_batch_workspace_bytes(d) > 0
    d[0].in_[0] = None
    with pytest.raises(bto.BtoError):
        bto.bto_batch_workspace_bytes(d)


@pytest.mark.parametrize("tile,ok", [(0, True), (16, True), (128, True), (1024, True), (8, False), (24, False),
                                     (1040, False), (-16, False)])
def test_panel_width_validation(tile, ok):
    descs = _batch([("bicgk", 100, 100)])
    if ok:
        assert bto.bto_batch_workspace_bytes(descs, tile) > 0
    else:
        with pytest.raises(bto.BtoError) as e:
            bto.bto_batch_workspace_bytes(descs, tile)
        assert e.value.arg == 3


# ---- the sweep's assignment of work items to blocks (bto_debug_lpt)
def _lpt(cost, grid):
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    block = np.full(len(cost), -1, dtype=np.int32)
    bto.bto_debug_lpt(len(cost), cost.ctypes.data, grid, block.ctypes.data)
    return block


def test_lpt_hand_worked_example():
    # Costs 9, 7, 6, 5, 4, 3, 1 over three blocks, worked by hand: 9, 7 and 6
    # open the blocks; 5 joins the least loaded (block 2: 6 -> 11); 4 joins
    # block 1 (7 -> 11); 3 joins block 0 (9 -> 12); 1 finds blocks 1 and 2
    # tied at 11 and takes the lower (block 1 -> 12).  Loads 12, 12, 11.
    assert _lpt([9, 7, 6, 5, 4, 3, 1], 3).tolist() == [0, 1, 2, 2, 1, 0, 1]


def test_lpt_equal_items_are_dealt_round_robin():
    assert np.array_equal(_lpt(np.full(1000, 2.5), 152), np.arange(1000) % 152)


def test_lpt_short_lists_take_one_block_each():
    assert _lpt([5.0, 4.0, 1.0], 8).tolist() == [0, 1, 2]
    assert _lpt([], 8).tolist() == []


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lpt_balance_bound(seed):
    # Each item goes to the least loaded block, so the busiest block exceeds
    # the least busy one by at most the largest item, and the mean by at most
    # (1 - 1/G) of it (Graham's bound for list scheduling).
    rng = np.random.default_rng(seed)
    cost = np.sort(np.exp(rng.uniform(np.log(1e3), np.log(4e6), 4096)))[::-1]
    G = 152
    block = _lpt(cost, G)
    assert block.min() >= 0 and block.max() < G
    load = np.bincount(block, weights=cost, minlength=G)
    assert load.max() - load.min() <= cost.max() * (1 + 1e-12)
    assert load.max() <= load.sum() / G + (1 - 1 / G) * cost.max() * (1 + 1e-12)


def test_lpt_validation():
    with pytest.raises(bto.BtoError) as e:
        _lpt([1.0, 2.0], 4)          # not in decreasing order
    assert e.value.status == _lib.BTO_ERR_INVALID_VALUE and e.value.arg == 2
    with pytest.raises(bto.BtoError) as e:
        _lpt([2.0, 1.0], 0)
    assert e.value.arg == 3
