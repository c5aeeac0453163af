"""Batched 1D-1V cases (dvm_batch_*) against the oracle, case by case.

Every case of a small uneven batch (different N_x, N_v, tau, p, boundary rule) must
match the FP64 oracle run on that case alone: 1e-12 (FP64 build) and 1e-5 (FP32
build) on moments, the same error scale as tests/test_gpu_parity.py.
"""
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
    cases = W.batched_tubes(ncases=24, steps=3, nx_range=(60, 300))
    a = dvm.Batch(cases, precision=dvm.F32)
    b = dvm.Batch(cases, precision=dvm.F32)
    U0 = a.pack([conserved(c) for c in cases])
    a.set_moments(U0)
    b.set_moments(U0)
    a.step(2)
    b.step(2)
    threads, cpt, ms = b.autotune()
    assert threads in (64, 128, 256) and cpt in (1, 2) and ms > 0
    a.step(3)
    b.step(3)
    assert np.array_equal(a.moments(), b.moments())
    assert np.array_equal(a.f(5), b.f(5))


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
