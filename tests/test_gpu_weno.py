"""GPU HOFKS with the WENO5 Euler solver (Section 4.3.3) against the oracle, through
the C ABI: moments, U_E / U_M / U_* and the sub-step count, FP64 at 1e-12 and FP32
at 1e-5 (the tolerances of tests/test_gpu_parity.py), in 1D (periodic and outflow),
2D and 3D; and the higher order of the WENO solver on the GPU itself."""
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


CASES = {
    "wave_1d": (lambda: W.entropy_wave_1d(64, tau=1e-3), 4),
    "sod_1d_outflow": (lambda: W.sod_1d(nx=120, nv=32, tau=1e-4), 5),
    "quadrant_2d": (lambda: W.quadrant_2d(n=29, nv=12, tau=1e-3, steps=3, dv=0.9), 3),
    "wave_3d": (lambda: W.density_wave_3d(n=10, nv=8, tau=1e-3, steps=2, dv=1.2), 2),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-12), (dvm.F32, 1e-5)])
def test_weno_hofks_matches_the_oracle(name, precision, tol):
    make, steps = CASES[name]
    case = make()
    orc = oracle.Scheme(grid(case, oracle.HOFKS_WENO), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(steps)
    s = dvm.Solver.from_case(case, precision=precision, scheme=dvm.HOFKS_WENO)
    s.set_moments(conserved(case))
    s.step(steps)
    assert moment_err(s.moments(), orc.moments()) <= tol
    Uo = orc.moments()
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    for a, b in zip(s.parts(), orc.parts()):
        assert (np.abs(a - b).max(axis=1) / scale).max() <= tol
    if precision == dvm.F64:
        assert s.info()["m"] == orc.info()["m"]
        fo = orc.f()
        assert np.abs(s.f() - fo).max() <= 1e-12 * np.abs(fo).max()


def test_weno_conserves_on_the_gpu():
    case = W.quadrant_2d(n=40, nv=16, tau=1e-3, steps=5, dv=0.8)
    s = dvm.Solver.from_case(case, precision=dvm.F64, scheme=dvm.HOFKS_WENO)
    U0 = conserved(case)
    s.set_moments(U0)
    s.step(5)
    scale = np.abs(U0).sum(1)
    scale[1:3] = scale[0]
    assert np.all(np.abs(s.moments().sum(1) - U0.sum(1)) <= 1e-13 * scale)


def test_weno_order_on_the_gpu_exceeds_muscl():
    """Fluid limit (tau = 0), dt_E ~ dx^2: on the GPU, FP64, the WENO solver's L1
    density error on the smooth entropy wave falls at rate > 4.5 and MUSCL's at ~2."""
    errs = {}
    for scheme in (dvm.HOFKS, dvm.HOFKS_WENO):
        e = []
        for nx in (20, 40, 80):
            case = W.entropy_wave_1d(nx, tau=0.0)
            s = dvm.Solver.from_case(case, precision=dvm.F64, scheme=scheme, subcycles=nx // 2)
            s.set_moments(conserved(case))
            s.step(case.steps)
            x = (np.arange(nx) + 0.5) / nx
            exact = 1 + 0.2 * np.sin(2 * np.pi * (x - 0.5 * case.extra["t_final"]))
            e.append(np.abs(s.moments()[0] - exact).sum() / np.abs(exact).sum())
            s.close()
        errs[scheme] = np.array(e)
    rw = np.log2(errs[dvm.HOFKS_WENO][:-1] / errs[dvm.HOFKS_WENO][1:])
    rm = np.log2(errs[dvm.HOFKS][:-1] / errs[dvm.HOFKS][1:])
    assert np.all(rw > 4.5) and np.all(rm < 2.3), (rw, rm)


def test_batch_rejects_the_weno_scheme():
    with pytest.raises(dvm.DvmError) as e:
        dvm.Batch([W.sod_1d(nx=20, nv=16)], precision=dvm.F64, scheme=dvm.HOFKS_WENO)
    assert e.value.code == dvm.ERR_ARG
