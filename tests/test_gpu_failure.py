"""Device-side failure detection without a GPU fault: the library's bounded
waits give up with DVM_ERR_TIMEOUT in the status word when the event they
wait for never comes (a block that never reaches the grid barrier, an
mbarrier nobody arrives at), and the context stays usable afterwards."""
import numpy as np
import pytest

import oracle
from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved, grid

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm  # noqa: E402


@pytest.mark.parametrize("which", [dvm.SELFTEST_GRID_BARRIER, dvm.SELFTEST_MBARRIER])
def test_bounded_wait_reports_timeout_and_context_survives(which):
    assert dvm.selftest_timeout(which) == dvm.ERR_TIMEOUT
    # the context still works: a small step against the oracle
    case = W.quadrant_2d(n=16, nv=8, tau=1e-3, steps=2, dv=1.0)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_moments(conserved(case))
    s.step(2)
    o = oracle.Scheme(grid(case), tau=case.tau)
    o.set_moments(conserved(case))
    o.step(2)
    Ug, Uo = s.moments(), o.moments()
    assert np.abs(Ug - Uo).max() <= 1e-12 * max(1.0, np.abs(Uo).max())
    s.close()


def test_selftest_rejects_unknown_case():
    with pytest.raises(dvm.DvmError):
        dvm.selftest_timeout(7)
