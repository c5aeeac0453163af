"""Batched cases (dvm_batch_*) against the oracle, case by case.

Every case of a small uneven batch (different dimension, N_x, N_v, tau, p, boundary
rule) must match the FP64 oracle run on that case alone: 1e-12 (FP64 build) and 1e-5
(FP32 build) on moments, the same error scale as tests/test_gpu_parity.py.
"""
import dataclasses

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


def small_batch():
    cases = [
        W.sod_1d(nx=37, nv=16, tau=1e-4, steps=4, dv=0.8),
        W.sod_1d(nx=100, nv=32, tau=1e-2, steps=4),
        W.sod_1d(nx=203, nv=24, tau=3e-3, steps=4, dv=0.55, left=(0.7, 0.9), right=(0.2, 0.3)),
        W.sod_1d(nx=64, nv=32, tau=np.inf, steps=4),
        W.sod_1d(nx=150, nv=20, tau=1e-5, steps=4, dv=0.7, p=2),
        W.entropy_wave_1d(80, nv=32, tau=1e-3),
    ]
    return cases


def run_oracle(case, steps, scheme):
    o = oracle.Scheme(grid(case, scheme), tau=case.tau)
    o.set_moments(conserved(case))
    o.step(steps)
    return o


@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-12), (dvm.F32, 1e-5)])
@pytest.mark.parametrize("scheme", [dvm.HOFKS, dvm.FKS])
def test_batch_cases_match_the_oracle(precision, tol, scheme):
    cases = small_batch()
    b = dvm.Batch(cases, precision=precision, scheme=scheme)
    b.set_moments(b.pack([conserved(c) for c in cases]))
    steps = 4
    b.step(steps)
    U = b.moments()
    for i, c in enumerate(cases):
        o = run_oracle(c, steps, scheme)
        assert moment_err(b.case_moments(U, i), o.moments()) <= tol, i
        if precision == dvm.F64:
            fo = o.f()
            assert np.abs(b.f(i) - fo).max() <= 1e-12 * np.abs(fo).max(), i


def test_batch_euler_substeps_match_the_oracle():
    cases = small_batch()
    b = dvm.Batch(cases, precision=dvm.F64)
    b.set_moments(b.pack([conserved(c) for c in cases]))
    b.step(2)
    info = b.info()
    assert info["n"] == 2
    for i, c in enumerate(cases):
        o = run_oracle(c, 2, dvm.HOFKS)
        if np.isinf(c.tau):
            assert info["m"][i] == 0
        else:
            assert info["m"][i] == o.info()["m"], i


def test_autotune_keeps_the_trajectory():
    """The autotuner only changes the launch: the state it leaves is the one it found
    (f restored), and the trajectory after it equals the untuned one up to the FP64
    merge order of the velocity chunks' partial sums."""
    cases = W.batched_tubes(ncases=24, steps=3, nx_range=(60, 300))
    a = dvm.Batch(cases, precision=dvm.F32)
    b = dvm.Batch(cases, precision=dvm.F32)
    U0 = a.pack([conserved(c) for c in cases])
    a.set_moments(U0)
    b.set_moments(U0)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.f(5), b.f(5))
    threads, cpt, vch, occ, ms = b.autotune()
    assert threads in (64, 128, 256) and cpt in (1, 2) and vch in (1, 2, 4) and occ in (0, 2, 4)
    assert ms > 0
    assert np.array_equal(a.f(5), b.f(5)) and np.array_equal(a.moments(), b.moments())
    a.step(3)
    b.step(3)
    assert moment_err(b.moments(), a.moments()) <= 1e-6
    assert np.abs(a.f(5) - b.f(5)).max() <= 1e-6 * np.abs(a.f(5)).max()


def rect_quadrant(nx, ny, nv, tau, dv):
    """The four-quadrant problem on an nx x ny periodic grid (rows cut from the
    square one): a 2D case whose extents differ."""
    sq = W.quadrant_2d(n=max(nx, ny), nv=nv, tau=tau, steps=4, dv=dv)
    n = max(nx, ny)
    cut = lambda a: a.reshape(n, n)[:ny, :nx].ravel().copy()
    return dataclasses.replace(sq, nx=(nx, ny), rho=cut(sq.rho), T=cut(sq.T),
                               u=np.stack([cut(sq.u[0]), cut(sq.u[1])]), name="quadrant_rect")


def mixed_batch():
    """1D tubes and 2D periodic cases of uneven size, velocity count, tau and p in
    one batch."""
    q_p2 = W.quadrant_2d(n=15, nv=12, tau=2e-2, steps=4, dv=0.9)
    q_p2.p = 2
    return [
        W.sod_1d(nx=37, nv=16, tau=1e-4, steps=4, dv=0.8),
        W.quadrant_2d(n=24, nv=12, tau=1e-3, steps=4, dv=0.9),
        W.sod_1d(nx=100, nv=32, tau=1e-2, steps=4),
        rect_quadrant(21, 13, 16, 5e-2, 0.7),
        q_p2,
        W.quadrant_2d(n=12, nv=8, tau=np.inf, steps=4, dv=1.0),
        W.entropy_wave_1d(80, nv=32, tau=1e-3),
        W.quadrant_2d(n=9, nv=20, tau=1e-5, steps=4, dv=0.5),
    ]


@pytest.mark.parametrize("vchunks", [1, 4])
@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-12), (dvm.F32, 1e-5)])
@pytest.mark.parametrize("scheme", [dvm.HOFKS, dvm.FKS])
def test_mixed_1d_2d_batch_matches_the_oracle(precision, tol, scheme, vchunks):
    cases = mixed_batch()
    b = dvm.Batch(cases, precision=precision, scheme=scheme)
    assert b.rows == 4
    b.set_tiling(128, 1, vchunks, 0)
    b.set_moments(b.pack([conserved(c) for c in cases]))
    steps = 4
    b.step(steps)
    U = b.moments()
    info = b.info()
    for i, c in enumerate(cases):
        o = run_oracle(c, steps, scheme)
        assert moment_err(b.case_moments(U, i), o.moments()) <= tol, i
        # the rows a 1D case does not use stay zero
        assert np.all(U[c.d + 2:, b.offsets[i]:b.offsets[i + 1]] == 0.0)
        if precision == dvm.F64:
            fo = o.f()
            assert np.abs(b.f(i) - fo).max() <= 1e-12 * np.abs(fo).max(), i
            if scheme == dvm.HOFKS:
                assert info["m"][i] == (0 if np.isinf(c.tau) else o.info()["m"]), i


def test_mixed_batch_periodic_2d_cases_conserve():
    cases = [W.quadrant_2d(n=n, nv=nv, tau=t, steps=5, dv=0.8) for n, nv, t in
             ((16, 12, 1e-3), (23, 16, 1e-1), (11, 8, 1e-5))] + [W.entropy_wave_1d(48, nv=32, tau=1e-2)]
    b = dvm.Batch(cases, precision=dvm.F64)
    U0 = b.pack([conserved(c) for c in cases])
    b.set_moments(U0)
    b.step(5)
    U = b.moments()
    for i in range(len(cases)):
        tot0 = b.case_moments(U0, i).sum(1)
        tot = b.case_moments(U, i).sum(1)
        # momentum rows (zero totals here) on the scale of the mass
        scale = np.abs(b.case_moments(U0, i)).sum(1)
        scale[1:cases[i].d + 1] = scale[0]
        assert np.all(np.abs(tot - tot0) <= 1e-13 * scale), i


def test_batch_rejects_non_periodic_2d_cases():
    c = W.quadrant_2d(n=10, nv=8, tau=1e-3, steps=2, dv=1.0)
    c.bc = (W.OUTFLOW, W.PERIODIC)
    with pytest.raises(dvm.DvmError) as e:
        dvm.Batch([W.sod_1d(nx=20, nv=16), c], precision=dvm.F64)
    assert e.value.code == dvm.ERR_ARG


def test_batch_of_the_tube_workload_conserves_in_periodic_cases():
    cases = [W.entropy_wave_1d(n, nv=32, tau=t) for n, t in ((64, 1e-3), (96, 1e-1), (128, 1e-5))]
    b = dvm.Batch(cases, precision=dvm.F64)
    U0 = b.pack([conserved(c) for c in cases])
    b.set_moments(U0)
    b.step(5)
    U = b.moments()
    for i in range(3):
        tot0 = b.case_moments(U0, i).sum(1)
        tot = b.case_moments(U, i).sum(1)
        assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(b.case_moments(U0, i)).sum(1) + 1e-15)
