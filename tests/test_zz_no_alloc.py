"""bto_bicgk_noalloc: BICGK for callers that cannot allocate device memory
(a plugin whose host owns all device memory, a fixed device footprint,
loops that cannot afford cudaMalloc's possible device synchronization).
It keeps its partial sums in a fixed device array inside the library
instead of a caller workspace.  Checked through the C ABI against the
workspace entry point bto_bicgk on two calls in a row, and against the
oracle, at the largest size its array accepts, with the next size rejected.  This file is
collected last so a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1205_1098_gb300 as bto
import synth
from gpu_util import TOL64, Out, dev, p, relerr, sync, ws

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


def _reference(m, n, A, pv, rv):
    q, s = Out(m), Out(n)
    wk, nb = ws("bicgk", 0, m, n)
    bto.bto_bicgk(m, n, A, m, pv, rv, q.ptr(), s.ptr(), p(wk), nb, None)
    sync()
    return q.host(), s.host()


def test_noalloc_matches_workspace_entry_twice():
    for call, (m, n, seed) in enumerate([(1500, 1100, 21), (2049, 777, 22)]):
        A = dev(synth.matrix(seed, 0, m, n))
        pv, rv = dev(synth.vector(seed, 1, n)), dev(synth.vector(seed, 2, m))
        qr, sr = _reference(m, n, A, pv, rv)
        q, s = Out(m), Out(n)
        bto.bto_bicgk_noalloc(m, n, A, m, pv, rv, q.ptr(), s.ptr(), None)
        sync()
        qg, sg = q.host(), s.host()
        assert relerr(qg, qr) <= TOL64 and relerr(sg, sr) <= TOL64, call
        assert np.array_equal(qg, qr) and np.array_equal(sg, sr), call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    m = n = 8192
    need = bto.bto_workspace_bytes("bicgk", 0, m, n)
    assert need > (4 << 20)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_noalloc(m, n, 0, m, 0, 0, 0, 0, None)
    assert e.value.status == bto.BTO_ERR_WORKSPACE and e.value.arg in (1, 2)


def _largest_accepted_square():
    """The largest square n whose BICGK workspace fits the fixed array (every
    smaller n fits too), found on the host from the workspace query."""
    limit = 4 << 20
    last = 0
    for n in range(1, 6001):
        if bto.bto_workspace_bytes("bicgk", 0, n, n) > limit:
            return last, n
        last = n
    raise AssertionError("no square size exceeds the array up to 6000")


def test_noalloc_largest_accepted_size_and_the_next():
    n, over = _largest_accepted_square()
    assert n >= 1 and over == n + 1
    A64 = synth.matrix(23, 0, n, n)
    p64, r64 = synth.vector(23, 1, n), synth.vector(23, 2, n)
    A, pv, rv = dev(A64), dev(p64), dev(r64)
    q, s = Out(n), Out(n)
    bto.bto_bicgk_noalloc(n, n, A, n, pv, rv, q.ptr(), s.ptr(), None)
    sync()
    qo, so = O.bicgk(n, n, A64, p64, r64)
    assert relerr(q.host(), qo) <= TOL64 and relerr(s.host(), so) <= TOL64
    qr, sr = _reference(n, n, A, pv, rv)
    assert np.array_equal(q.host(), qr) and np.array_equal(s.host(), sr)
    with pytest.raises(bto.BtoError) as e:
        bto.bto_bicgk_noalloc(over, over, 0, over, 0, 0, 0, 0, None)
    assert e.value.status == bto.BTO_ERR_WORKSPACE


def test_noalloc_matches_the_oracle():
    m, n = 1777, 2049
    A64 = synth.matrix(24, 0, m, n)
    p64, r64 = synth.vector(24, 1, n), synth.vector(24, 2, m)
    q, s = Out(m), Out(n)
    bto.bto_bicgk_noalloc(m, n, dev(A64), m, dev(p64), dev(r64), q.ptr(), s.ptr(), None)
    sync()
    qo, so = O.bicgk(m, n, A64, p64, r64)
    assert relerr(q.host(), qo) <= TOL64 and relerr(s.host(), so) <= TOL64
