"""Section 5.4's 2D implosion and the Strang-split FKS of Section 4.2 on the GPU,
through the C ABI, against the FP64 oracle (tolerances of tests/test_gpu_parity.py:
1e-12 FP64, 1e-5 FP32 on moments; f element by element in FP64)."""
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


def moment_err(Ug, Uo):
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    return (np.abs(Ug - Uo).max(axis=1) / scale).max()


def run_both(case, steps, scheme, precision):
    o = oracle.Scheme(grid(case, scheme), tau=case.tau)
    o.set_moments(conserved(case))
    o.step(steps)
    s = dvm.Solver.from_case(case, precision=precision, scheme=scheme)
    s.set_moments(conserved(case))
    s.step(steps)
    return s, o


@pytest.mark.parametrize("scheme", [dvm.HOFKS, dvm.FKS])
@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-12), (dvm.F32, 1e-5)])
def test_implosion_matches_the_oracle(scheme, precision, tol):
    """40^2 x 30^2, outflow, p = 15 (t = 0.07 in 28 steps), the first 3 steps."""
    case = W.implosion_2d(40)
    s, o = run_both(case, 3, scheme, precision)
    assert moment_err(s.moments(), o.moments()) <= tol
    if precision == dvm.F64:
        fo = o.f()
        assert np.abs(s.f() - fo).max() <= 1e-12 * np.abs(fo).max()


def test_implosion_keeps_the_diagonal_symmetry():
    """The data and the velocity grid are the same in x and y: the density stays
    symmetric under x <-> y (up to the order of FP64 sums) over the whole run."""
    case = W.implosion_2d(40)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_moments(conserved(case))
    s.step(case.steps)
    rho = s.moments()[0].reshape(40, 40)
    assert np.abs(rho - rho.T).max() <= 1e-10 * rho.max()
    assert rho.max() > 1.1  # the colliding streams have compressed the gas


STRANG_CASES = {
    "quadrant_periodic": lambda: W.quadrant_2d(n=16, nv=16, tau=2e-2, steps=4, dv=0.7),
    "sod_outflow": lambda: W.sod_1d(nx=80, nv=32, tau=3e-3),
    "shear_taufield": lambda: W.shear_layer_2d(n=20, nv=10, steps=3, dv=1.0),
}


@pytest.mark.parametrize("name", list(STRANG_CASES))
@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-12), (dvm.F32, 1e-5)])
def test_strang_fks_matches_the_oracle(name, precision, tol):
    case = STRANG_CASES[name]()
    s, o = run_both(case, 4, dvm.FKS_STRANG, precision)
    assert moment_err(s.moments(), o.moments()) <= tol
    fo = o.f()
    assert np.abs(s.f() - fo).max() <= (1e-12 if precision == dvm.F64 else 1e-5) * np.abs(fo).max()
    # and its f differs from the first-order scheme's, its moments do not
    t = dvm.Solver.from_case(case, precision=precision, scheme=dvm.FKS)
    t.set_moments(conserved(case))
    t.step(4)
    assert moment_err(t.moments(), s.moments()) <= tol
    assert np.abs(t.f() - s.f()).max() > 1e-6 * np.abs(fo).max()


def test_strang_is_rejected_by_the_batch_and_the_learned_path():
    with pytest.raises(dvm.DvmError):
        dvm.Batch([W.sod_1d(nx=20, nv=16)], precision=dvm.F64, scheme=dvm.FKS_STRANG)
    case = W.quadrant_2d(n=12, nv=8, tau=1e-2, steps=2, dv=1.0)
    s = dvm.Solver.from_case(case, precision=dvm.F64, scheme=dvm.FKS_STRANG)
    s.set_moments(conserved(case))
    with pytest.raises(dvm.DvmError):
        s.learn_enable()
