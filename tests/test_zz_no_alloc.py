"""bto_bicgk_noalloc: BICGK for callers that cannot allocate device memory
(a plugin whose host owns all device memory, a fixed device footprint,
loops that cannot afford cudaMalloc's possible device synchronization).
It keeps its partial sums in a fixed device array inside the library
instead of a caller workspace.  Checked through the C ABI against the
workspace entry point bto_bicgk on two calls in a row.  This file is
collected last so a failure here leaves every other test already run."""
import numpy as np
import pytest
import torch

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
