"""The FP64 tile planner, checked on the host (bto_panel_plan touches no
device): every plan covers the matrix with panels at most 512 columns wide
and row blocks of at least one 2048-row chunk where the matrix has one;
fused GEMVER takes one chunk per row block (the schedule search's finding);
large problems get about two tiles per multiprocessor; overrides are
clamped as documented; and the documented limit of the no-allocation BICGK
(every square n up to 3427 on 152 multiprocessors fits its 4 MiB scratch)
holds.  The double-float forms' plan: panels of at most 1024 columns, at
most one tile per multiprocessor where that allows, one plan for every op,
and 8 x 19 tiles at the benchmarked n = 16384 on 152 multiprocessors."""
import itertools

import pytest

import paper_1205_1098_gb300 as bto
from paper_1205_1098_gb300 import build

OPS = ["bicgk", "atax", "gemver", "gesummv", "dgemv", "dgemvt"]
SIZES = [1, 2, 63, 64, 65, 100, 2047, 2048, 2049, 4096, 5000, 16384, 40000]


@pytest.fixture(scope="module", autouse=True)
def _lib_built():
    build.build()
    for op in OPS:
        for form in (0, 1):
            bto.bto_schedule_set(bto.OPS[op], form, 0, 0)


def ceil_div(a, b):
    return -(-a // b)


@pytest.mark.parametrize("sms", [152, 148, 132, 16])
def test_plans_cover_the_matrix(sms):
    for op, form, m, n in itertools.product(OPS, (0, 1), SIZES, SIZES):
        nr, nc = bto.bto_panel_plan(op, form, m, n, sms)
        assert 1 <= nc <= n and ceil_div(n, nc) <= 512, (op, form, m, n, nr, nc)
        assert 1 <= nr <= max(1, ceil_div(m, 64)), (op, form, m, n, nr, nc)
        # Row blocks are at least one chunk tall unless the matrix is shorter.
        assert nr <= max(1, ceil_div(m, 2048)), (op, form, m, n, nr, nc)


def test_empty_matrices_plan_no_tiles():
    for op in OPS:
        assert bto.bto_panel_plan(op, 0, 0, 100, 152) == (0, 0)
        assert bto.bto_panel_plan(op, 0, 100, 0, 152) == (0, 0)


def test_fused_gemver_takes_one_chunk_per_row_block():
    for m in (2048, 4096, 5000, 16384, 40000):
        nr, _ = bto.bto_panel_plan("gemver", 0, m, 16384, 152)
        assert nr == ceil_div(m, 2048), m
    # The unfused form keeps the general plan.
    assert bto.bto_panel_plan("gemver", 1, 16384, 16384, 152)[0] == 2


def test_large_problems_feed_two_blocks_per_multiprocessor():
    """About two tiles per multiprocessor: balanced panels may leave a few of
    the two-per-SM slots empty (n = 4096 on 132 SMs: 128 panels of 32
    columns x 2 row blocks), never more than a tenth."""
    for op, m, n, sms in itertools.product(OPS, (4096, 16384, 40000), (4096, 16384, 40000), (152, 132)):
        nr, nc = bto.bto_panel_plan(op, 0, m, n, sms)
        assert nr * nc >= 0.9 * 2 * sms, (op, m, n, sms, nr, nc)
    assert bto.bto_panel_plan("bicgk", 0, 16384, 16384, 152) == (2, 152)


def test_overrides_are_clamped():
    try:
        bto.bto_schedule_set(bto.OPS["dgemv"], 0, 1 << 20, 1 << 20)
        nr, nc = bto.bto_panel_plan("dgemv", 0, 1000, 700, 152)
        assert nc == 700                          # at most n panels
        assert nr <= ceil_div(1000, 64)           # at most one block per 64 rows
        bto.bto_schedule_set(bto.OPS["dgemv"], 0, 1, 1)
        nr, nc = bto.bto_panel_plan("dgemv", 0, 1000, 70000, 152)
        assert nc == ceil_div(70000, 512) and nr == 1   # panels stay at most 512 wide
        # The other form and the other ops keep their automatic plans.
        assert bto.bto_panel_plan("dgemv", 1, 1000, 70000, 152) != (1, ceil_div(70000, 512))
        assert bto.bto_panel_plan("bicgk", 0, 16384, 16384, 152) == (2, 152)
    finally:
        bto.bto_schedule_set(bto.OPS["dgemv"], 0, 0, 0)


def _bicgk_workspace(m, n, sms):
    nr, nc = bto.bto_panel_plan("bicgk", 0, m, n, sms)
    up = lambda x, a: ceil_div(x, a) * a
    ldq, lds = up(max(m, 1), 32), up(max(n, 1), 32)
    return 256 + up(nc * ldq * 8, 256) + up(nr * lds * 8, 256)


def test_noalloc_limit_holds():
    """bto_bicgk_noalloc accepts a problem whose BICGK workspace fits 4 MiB;
    its documentation promises every square n up to 3427 on 152
    multiprocessors."""
    limit = 4 << 20          # BTO_NOALLOC_SCRATCH_BYTES
    assert all(_bicgk_workspace(n, n, 152) <= limit for n in range(1, 3428))
    assert _bicgk_workspace(3428, 3428, 152) > limit


def test_plan_query_validation():
    for args, pos in ((("bicgk", 0, -1, 4, 152), 3), (("bicgk", 0, 4, -1, 152), 4), (("bicgk", 0, 4, 4, 0), 5),
                      ((9, 0, 4, 4, 152), 1), (("bicgk", 4, 4, 4, 152), 2)):
        with pytest.raises(bto.BtoError) as e:
            bto.bto_panel_plan(*args)
        assert e.value.arg == pos


DF_FORMS = (2, 3)   # BTO_FORM_DF, BTO_FORM_DF_UNFUSED


@pytest.mark.parametrize("sms", [152, 148, 16])
def test_df_plans_cover_the_matrix(sms):
    for op, form, m, n in itertools.product(OPS, DF_FORMS, SIZES, SIZES):
        nr, nc = bto.bto_panel_plan(op, form, m, n, sms)
        cu, ru = ceil_div(n, 16), ceil_div(m, 256)           # 16-column and 256-row units
        assert 1 <= nc <= cu and 1 <= nr <= ru, (op, form, m, n, nr, nc)
        assert ceil_div(cu, nc) * 16 <= 1024, (op, form, m, n, nr, nc)
        if ceil_div(cu, 64) <= sms:
            assert nr * nc <= sms, (op, form, m, n, nr, nc)   # at most one tile per block
        assert (nr, nc) == bto.bto_panel_plan("bicgk", 2, m, n, sms)


def test_df_plan_at_the_benchmarked_size():
    # n = 16384 on 152 multiprocessors: 8 row blocks of 2048 rows and 19
    # panels of at most 54 units of 16 columns.
    assert bto.bto_panel_plan("bicgk", 2, 16384, 16384, 152) == (8, 19)
    assert bto.bto_panel_plan("gemver", 3, 16384, 16384, 152) == (8, 19)
