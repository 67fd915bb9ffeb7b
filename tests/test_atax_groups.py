"""ATAX / BATAX group-band kernel: shapes that exercise its plan against the
oracle.  Groups grow past 16 blocks when n exceeds 16 x 4096 columns (and
groups beyond the band count stay idle); beyond 4096 columns per block on
every SM the two-pass form (t = A x through the workspace) runs instead;
bands of fewer than 16 rows, odd leading dimensions (scalar loads) and
integer inputs (exact) are covered too."""
import numpy as np
import pytest

from f64_cases import run_atax
from gpu_util import TOL64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1205_1098_gb300 import build
    build.build()


@pytest.mark.parametrize("shape", [(17, 33, 17), (16, 4096, 16), (40, 70001, 40), (3, 1300000, 3),
                                   (4112, 2000, 4113), (31, 2, 31)],
                         ids=lambda s: "%dx%d_ld%d" % s)
def test_atax_plan_shapes(shape):
    m, n, lda = shape
    for name, (g, o) in run_atax(m, n, lda, 0).items():
        nr = np.linalg.norm(o)
        assert np.linalg.norm(g - o) <= TOL64 * nr, name


@pytest.mark.parametrize("shape", [(40, 70001, 40), (1000, 3001, 1001), (3, 1300000, 3)],
                         ids=lambda s: "%dx%d_ld%d" % s)
def test_atax_plan_shapes_integer_exact(shape):
    m, n, lda = shape
    for name, (g, o) in run_atax(m, n, lda, 1, beta=2.0).items():
        assert np.array_equal(g, o), name
