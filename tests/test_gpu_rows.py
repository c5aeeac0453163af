"""The row pass (whole x rows moved by tensor copies through shared memory,
opt-in with DVM_ROWS_PASS=1) against the FP64 oracle.

* 2D-2V quadrant, 64^2 x 16^2: HOFKS and FKS, FP32, 1e-5 on the moments;
* 3D-3V density wave, 32^3 x 8^3, HOFKS, FP32, 1e-5;
* learned path with a seeded flag mask (flagged targets keep their pieces);
* the row pass and the windowed pass on the same 128^2 x 32^2 run agree to
  FP32 rounding;
* enough steps that the transported rows wrap around N_y inside a block
  (single-row copies) as well as not (copies of Y rows).
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


@pytest.fixture(autouse=True)
def rows_pass(monkeypatch):
    monkeypatch.setenv("DVM_ROWS_PASS", "1")


def both(case, steps, scheme=None, flags=None):
    s = dvm.Solver.from_case(case, precision=dvm.F32, scheme=scheme)
    assert s.kinetic_kernel() == "rows"
    s.set_moments(conserved(case))
    o = oracle.Scheme(grid(case, scheme), tau=case.tau)
    o.set_moments(conserved(case))
    if flags is not None:
        s.learn_enable(dvm.LEARN_GIVEN)
        s.learn_set_flags(flags)
        for _ in range(steps):
            o.step_flagged(flags)
    else:
        o.step(steps)
    s.step(steps)
    U = s.moments()
    s.close()
    return U, o.moments()


@pytest.mark.parametrize("scheme", [None, "fks"])
def test_rows_2d_matches_oracle(scheme):
    case = W.quadrant_2d(n=64, nv=16, tau=1e-3, steps=5, dv=0.7)
    sch = None if scheme is None else dvm.FKS
    Ug, Uo = both(case, 5, scheme=sch)
    assert moment_err(Ug, Uo) <= 1e-5


def test_rows_3d_matches_oracle():
    case = W.density_wave_3d(n=32, nv=8, tau=1e-4, steps=3, dv=1.2)
    Ug, Uo = both(case, 3)
    assert moment_err(Ug, Uo) <= 1e-5


def test_rows_learned_flags_match_oracle():
    case = W.shear_layer_2d(n=64, nv=16, steps=3, dv=0.8)
    fl = blocky_flags(np.random.default_rng(5), case.nx, 0.5, 8)
    Ug, Uo = both(case, 3, flags=fl)
    assert moment_err(Ug, Uo) <= 1e-5


def test_rows_and_window_agree(monkeypatch):
    case = W.quadrant_2d(n=128, nv=32, tau=1e-3, steps=6)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("DVM_ROWS_PASS", mode)
        s = dvm.Solver.from_case(case, precision=dvm.F32)
        out[mode] = s.kinetic_kernel()
        s.set_moments(conserved(case))
        s.step(6)
        out["U" + mode] = s.moments()
        s.close()
    assert out["1"] == "rows" and out["0"] == "window"
    assert moment_err(out["U1"], out["U0"]) <= 2e-6
