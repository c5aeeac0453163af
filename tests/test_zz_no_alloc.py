"""The allocation-free entry point (dvm_equilibrium_noalloc) against the normal path.

Some callers cannot allocate device memory at all (a program confined to a memory
budget fixed in advance, or a host thread that must stay out of the CUDA
allocator); for them libdvm offers one entry point whose scratch is a static
device array.  Its output must equal what the allocating path produces: the
f^0 = E[U] that dvm_set_state_moments builds and dvm_get_f returns at step 0.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm  # noqa: E402


def reference_f(case, U):
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_moments(U)
    return s.f()


def noalloc_f(case, U):
    cfg, keep = dvm.config_from_case(case, precision=dvm.F64)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    fd = torch.full((case.nvel, case.ncells), float("nan"), dtype=torch.float64, device="cuda")
    rc = dvm.equilibrium_noalloc(cfg, Ud, fd)
    assert rc == 0, rc
    return fd.cpu().numpy()


# the scratch array and its fixed header (include/dvm.h); the per-cell
# parameters take 8 (P + 1) bytes a cell, P = 16 rows in 2D and 3D
SCRATCH_BYTES = 8 << 20
HEADER_BYTES = 512
MAX_CELLS_2D_3D = (SCRATCH_BYTES - HEADER_BYTES) // (8 * 17)   # 61677


def test_noalloc_equilibrium_matches_the_allocating_path_twice_in_a_row():
    """Two calls in a row on different problems: the second must not see the first
    call's scratch contents."""
    a = W.quadrant_2d(n=40, nv=12, tau=1e-3, steps=1, dv=0.9)
    b = W.density_wave_3d(n=9, nv=8, tau=1e-4, steps=1, dv=1.2)
    for case in (a, b, a):
        U = conserved(case)
        want = reference_f(case, U)
        got = noalloc_f(case, U)
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_noalloc_3d_near_the_cell_limit_matches_the_allocating_path():
    """A 3D problem close to the scratch limit (39^3 = 59319 cells, about 230
    blocks per kernel): the per-cell parameters fill almost the whole array, and
    blocks that run after cell 0's parameters are written still read the 5 x 5
    (C C^T)^{-1}, so any overlap of the two regions shows in f.  Twice in a row."""
    case = W.density_wave_3d(n=39, nv=6, tau=1e-4, steps=1, dv=1.2)
    assert case.ncells <= MAX_CELLS_2D_3D
    U = conserved(case)
    want = reference_f(case, U)
    for _ in range(2):
        got = noalloc_f(case, U)
        assert np.all(np.isfinite(got))
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_noalloc_rejects_problems_beyond_its_scratch():
    for case in (W.quadrant_2d(n=249, nv=8, tau=1e-3, steps=1),      # 62001 cells
                 W.density_wave_3d(n=40, nv=6, tau=1e-4, steps=1)):  # 64000 cells
        assert case.ncells > MAX_CELLS_2D_3D
        cfg, keep = dvm.config_from_case(case, precision=dvm.F64)
        U = torch.zeros((case.d + 2, case.ncells), dtype=torch.float64, device="cuda")
        f = torch.zeros((case.nvel, case.ncells), dtype=torch.float64, device="cuda")
        assert dvm.equilibrium_noalloc(cfg, U, f) == dvm.ERR_TOO_LARGE
    # the largest accepted 2D grid is not rejected
    case = W.quadrant_2d(n=248, nv=8, tau=1e-3, steps=1, dv=0.9)     # 61504 cells
    U = conserved(case)
    want = reference_f(case, U)
    assert np.abs(noalloc_f(case, U) - want).max() <= 1e-12 * np.abs(want).max()


def test_noalloc_reports_nonphysical_moments():
    case = W.sod_1d(nx=30, nv=16)
    U = conserved(case)
    U[0, 4] = -1.0
    cfg, keep = dvm.config_from_case(case, precision=dvm.F64)
    Ud = torch.from_numpy(U).cuda()
    f = torch.zeros((case.nvel, case.ncells), dtype=torch.float64, device="cuda")
    assert dvm.equilibrium_noalloc(cfg, Ud, f) == dvm.ERR_NONPHYSICAL
    # and the next call on good data is clean again (status word cleared per call)
    good = W.sod_1d(nx=30, nv=16)
    assert np.abs(noalloc_f(good, conserved(good)) - reference_f(good, conserved(good))).max() \
        <= 1e-12
