"""Parity at the full workload sizes, in the launch configuration bench.py times.

* 2D-2V quadrant, 256^2 x 32^2, FP32 (windowed pass, staged loads, forked Euler
  kernel): two steps against the FP64 oracle at the full size (1e-5 on moments,
  same sub-step count).
* 3D-3V density wave, 96^3 x 24^3, FP32: too large for the oracle; checked by
  properties that hold at any size: periodic totals conserved, rho > 0, theta > 0.
* 512 batched tubes: the whole batch advanced together, a seeded sample of tubes
  against the oracle run on each tube alone (1e-5).
* Learned path, 512^2 x 32^2 shear layer, FP32: one step with a seeded flag mask
  against the oracle's flagged step at the full size.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved, grid
from tests.test_oracle_learned import blocky_flags

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm  # noqa: E402


def moment_err(Ug, Uo):
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    return (np.abs(Ug - Uo).max(axis=1) / scale).max()


def test_quadrant_256_full_size_matches_oracle():
    case = W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=2)
    s = dvm.Solver.from_case(case, precision=dvm.F32)
    s.set_moments(conserved(case))
    s.step(2)
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(2)
    assert moment_err(s.moments(), orc.moments()) <= 1e-5
    assert s.info()["m"] == orc.info()["m"]


def test_density_wave_96_full_size_conserves_and_stays_physical():
    case = W.density_wave_3d(n=96, nv=24, tau=1e-4, steps=2)
    U0 = conserved(case)
    s = dvm.Solver.from_case(case, precision=dvm.F32)
    s.set_moments(U0)
    s.step(2)
    U = s.moments()
    scale = np.abs(U0).sum(1)
    scale[1:4] = scale[0]
    assert np.all(np.abs(U.sum(1) - U0.sum(1)) <= 1e-6 * scale)
    rho = U[0]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / rho
    theta = (U[4] - ke) / (1.5 * rho)
    assert rho.min() > 0 and theta.min() > 0
    # the density wave is advected, not destroyed: its amplitude is kept
    assert 0.9 * 0.2 < (rho.max() - rho.min()) / 2 < 1.1 * 0.2


def test_all_512_tubes_match_the_oracle_on_a_sample():
    cases = W.batched_tubes(ncases=512, steps=2)
    b = dvm.Batch(cases, precision=dvm.F32)
    b.set_moments(b.pack([conserved(c) for c in cases]))
    b.step(2)
    U = b.moments()
    rng = np.random.default_rng(1212)
    for i in rng.choice(len(cases), 8, replace=False):
        c = cases[i]
        o = oracle.Scheme(grid(c), tau=c.tau)
        o.set_moments(conserved(c))
        o.step(2)
        assert moment_err(b.case_moments(U, i), o.moments()) <= 1e-5, i


def test_learned_step_512_full_size_matches_oracle():
    case = W.shear_layer_2d(n=512, nv=32, steps=1, dv=0.4)
    fl = blocky_flags(np.random.default_rng(7), case.nx, 0.6, 64)
    s = dvm.Solver.from_case(case, precision=dvm.F32)
    s.set_moments(conserved(case))
    s.learn_enable(dvm.LEARN_GIVEN)
    s.learn_set_flags(fl)
    s.step(1)
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step_flagged(fl)
    assert moment_err(s.moments(), orc.moments()) <= 1e-5
