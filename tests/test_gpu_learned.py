"""Learned regime path on the GPU against the oracle (through the C ABI).

The flagged step (lambda -> 0 form of Theorem 1 at flagged cells) is compared
with the oracle's ``step_flagged`` on the same seeded flag masks: 1e-12 on
moments and f in the FP64 build (generic kinetic pass), 1e-5 on moments in the
FP32 build (windowed pass, with whole flagged tiles skipped).  Features, labels
and the one-step check are compared with the oracle's definitions; the
network's FP32 forward pass and gradient with the FP64 oracle network.
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


def shear_case(n=40, nv=12, dv=0.9, steps=3):
    """2D shear layer with a seeded smooth tau field (fluid and rarefied zones)."""
    c = W.shear_layer_2d(n=n, nv=nv, steps=steps, dv=dv, width=0.08)
    return c


def masks(case, nsteps, seed=31, block=8, frac=0.7):
    rng = np.random.default_rng(seed)
    return [blocky_flags(rng, case.nx, frac, block) for _ in range(nsteps)]


def run_pair(case, precision, fl_list):
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    s = dvm.Solver.from_case(case, precision=precision)
    s.set_moments(conserved(case))
    s.learn_enable(dvm.LEARN_GIVEN)
    for fl in fl_list:
        s.learn_set_flags(fl)
        s.step(1)
        orc.step_flagged(fl)
    return s, orc


def effective(fl, case):
    lam = np.exp(-case.dt / np.broadcast_to(case.tau, (case.ncells,)))
    return (fl != 0) & (lam != 1.0)


def test_flagged_steps_match_oracle_fp64():
    case = shear_case(n=24, nv=10, dv=1.0)
    fls = masks(case, 4, block=4, frac=0.6)
    s, orc = run_pair(case, dvm.F64, fls)
    assert moment_err(s.moments(), orc.moments()) <= 1e-12
    fo = orc.f()
    assert np.abs(s.f() - fo).max() <= 1e-12 * np.abs(fo).max()
    assert np.array_equal(s.learn_flags() != 0, effective(fls[-1], case))


def test_flagged_steps_match_oracle_fp32_windowed():
    """nv = 16 (a multiple of 8), periodic, p = 1: the windowed pass, with CTAs
    whose targets and sources are all flagged skipped."""
    case = shear_case(n=48, nv=16, dv=0.7)
    fls = masks(case, 4, block=16, frac=0.75)
    s, orc = run_pair(case, dvm.F32, fls)
    assert moment_err(s.moments(), orc.moments()) <= 1e-5
    fo = orc.f()
    assert np.abs(s.f() - fo).max() <= 1e-5 * np.abs(fo).max()


def test_flagged_1d_outflow_matches_oracle():
    case = W.sod_1d(nx=120, nv=32, tau=1e-3)
    rng = np.random.default_rng(4)
    fls = [blocky_flags(rng, case.nx, 0.5, 10) for _ in range(5)]
    s, orc = run_pair(case, dvm.F64, fls)
    assert moment_err(s.moments(), orc.moments()) <= 1e-12
    fo = orc.f()
    assert np.abs(s.f() - fo).max() <= 1e-12 * np.abs(fo).max()


def test_learned_periodic_run_conserves():
    case = shear_case(n=32, nv=12, dv=0.9)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    U0 = conserved(case)
    s.set_moments(U0)
    s.learn_enable(dvm.LEARN_GIVEN)
    for fl in masks(case, 5, seed=9, block=8):
        s.learn_set_flags(fl)
        s.step(1)
    tot0, tot = U0.sum(1), s.moments().sum(1)
    assert np.all(np.abs(tot - tot0) <= 1e-13 * np.abs(U0).sum(1).max())


def test_disable_writes_back_equilibria():
    """Switching the path off stores f = E[U] into the flagged cells' pieces:
    the following plain steps equal the oracle's plain steps from that state."""
    case = shear_case(n=24, nv=10, dv=1.0)
    fls = masks(case, 2, block=4)
    s, orc = run_pair(case, dvm.F64, fls)
    s.learn_disable()
    s.step(2)
    orc.step(2)
    assert moment_err(s.moments(), orc.moments()) <= 1e-12
    fo = orc.f()
    assert np.abs(s.f() - fo).max() <= 1e-12 * np.abs(fo).max()


def test_features_match_oracle():
    case = shear_case(n=32, nv=12, dv=0.9)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_moments(conserved(case))
    s.step(2)
    U = s.moments()
    got = s.features().T.astype(np.float64)
    want = oracle.features(grid(case), U, case.tau)
    np.testing.assert_allclose(got[:4], want[:4], rtol=2e-6, atol=1e-6)
    np.testing.assert_allclose(got[4], want[4], atol=1e-5)
    away = want[5:] > -11.0
    assert np.abs(got[5:][away] - want[5:][away]).max() <= 1e-4
    assert np.all(got[5:][~away] <= -10.0)


@pytest.mark.parametrize("flagged", [False, True])
def test_noneq_label_matches_oracle(flagged):
    case = shear_case(n=24, nv=10, dv=1.0)
    if flagged:
        s, orc = run_pair(case, dvm.F64, masks(case, 2, block=4))
    else:
        s = dvm.Solver.from_case(case, precision=dvm.F64)
        s.set_moments(conserved(case))
        s.step(3)
        orc = oracle.Scheme(grid(case), tau=case.tau)
        orc.set_moments(conserved(case))
        orc.step(3)
    got = s.noneq().astype(np.float64)
    want = oracle.noneq(grid(case), orc.f(), orc.moments())
    hi = want > -9.0
    assert np.abs(got[hi] - want[hi]).max() <= 1e-5
    assert np.all(got[~hi] <= -8.5)


def test_one_step_check_matches_oracle():
    """dvm_learn_step_checked: the check values of given cells equal the oracle's
    raw one-step non-equilibrium, and the step itself the oracle's flagged step."""
    case = shear_case(n=24, nv=10, dv=1.0)
    fls = masks(case, 2, block=4)
    s, orc = run_pair(case, dvm.F64, fls[:1])
    fl = fls[1]
    cells = np.concatenate([np.flatnonzero(fl)[:40], np.flatnonzero(fl == 0)[:10]])
    s.learn_set_flags(fl)
    got = s.learn_step_checked(cells).astype(np.float64)
    raw = orc.clone()
    raw.step_flagged(fl, keep_raw=True)
    orc.step_flagged(fl)
    want = oracle.noneq(grid(case), raw.f(), raw.moments())[cells]
    assert np.abs(got - want).max() <= 1e-5, np.abs(got - want).max()
    assert moment_err(s.moments(), orc.moments()) <= 1e-12


def test_mlp_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(21)
    P = (rng.standard_normal(dvm.MLP_NPARAM) * 0.3).astype(np.float32)
    X = rng.standard_normal((777, 10)).astype(np.float32)
    y = rng.standard_normal(777).astype(np.float32)
    m = dvm.Mlp(dvm.F32)
    m.set_params(P)
    got = m.forward(X).cpu().numpy().astype(np.float64)
    want = oracle.mlp_forward(P.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-5)
    loss, g = m.loss_grad(X, y)
    lo, go = oracle.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - lo) <= 1e-6 * lo
    assert np.linalg.norm(g - go) <= 1e-6 * np.linalg.norm(go), np.linalg.norm(g - go) / np.linalg.norm(go)


def test_training_lowers_the_loss():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20000, 10)).astype(np.float32)
    y = (np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.1 * X[:, 7]).astype(np.float32)
    P0 = (rng.standard_normal(dvm.MLP_NPARAM) * 0.1).astype(np.float32)
    m = dvm.Mlp(dvm.F32)
    m.set_params(P0)
    l0, _ = m.loss_grad(X, y)
    l1 = m.train(X, y, epochs=8, batch=512, lr=3e-3)
    l2, _ = m.loss_grad(X, y)
    assert l2 < 0.2 * l0, (l0, l1, l2)


def test_mlp_mode_flags_follow_the_network():
    """MLP mode: the flag of each cell is (prediction < thr); the prediction is the
    network on the normalised features (compared with the oracle's FP64 network
    on the oracle's features)."""
    case = shear_case(n=32, nv=12, dv=0.9)
    s = dvm.Solver.from_case(case, precision=dvm.F32)
    s.set_moments(conserved(case))
    s.step(1)
    U = s.moments()
    rng = np.random.default_rng(8)
    P = (rng.standard_normal(dvm.MLP_NPARAM) * 0.2).astype(np.float32)
    F = oracle.features(grid(case), U, case.tau)
    shift = F.mean(1)
    scale = 1.0 / (F.std(1) + 1e-6)
    thr = 0.0
    s.learn_enable(dvm.LEARN_MLP, thr=thr, check_every=1, check_samples=64, shift=shift,
                   scale=scale)
    s.learn_set_params(P)
    s.step(1)
    pred = s.learn_predictions().astype(np.float64)
    Xn = ((F.T - shift.astype(np.float32)) * scale.astype(np.float32)).astype(np.float64)
    want = oracle.mlp_forward(P.astype(np.float64), Xn)
    np.testing.assert_allclose(pred, want, rtol=1e-3, atol=1e-3)
    fl = s.learn_flags() != 0
    assert np.array_equal(fl, pred < thr)
    st = s.learn_stats()
    assert st["steps"] == 1 and st["checks"] == 1 and st["flagged"] == fl.sum()


def test_tensor_core_forward_matches_oracle():
    """BF16 operands, FP32 accumulate (tcgen05): within BF16 rounding of the FP64
    network (inputs, weights and the hidden layer carry 8-bit mantissas)."""
    rng = np.random.default_rng(23)
    P = (rng.standard_normal(dvm.MLP_NPARAM) * 0.3).astype(np.float32)
    X = rng.standard_normal((1000, 10)).astype(np.float32)  # 7 full tiles + a ragged one
    m = dvm.Mlp(dvm.BF16S)
    m.set_params(P)
    got = m.forward(X).cpu().numpy().astype(np.float64)
    want = oracle.mlp_forward(P.astype(np.float64), X.astype(np.float64))
    err = np.abs(got - want)
    assert err.max() <= 0.03 * max(1.0, np.abs(want).max()), err.max()
    assert np.corrcoef(got, want)[0, 1] > 0.9999


def test_mlp_mode_with_tensor_core_network():
    case = shear_case(n=40, nv=12, dv=0.9)
    s = dvm.Solver.from_case(case, precision=dvm.F32)
    s.set_moments(conserved(case))
    s.step(1)
    U = s.moments()
    rng = np.random.default_rng(8)
    P = (rng.standard_normal(dvm.MLP_NPARAM) * 0.2).astype(np.float32)
    F = oracle.features(grid(case), U, case.tau)
    shift, scale = F.mean(1), 1.0 / (F.std(1) + 1e-6)
    s.learn_enable(dvm.LEARN_MLP, mlp_precision=dvm.BF16S, thr=0.0, shift=shift, scale=scale)
    s.learn_set_params(P)
    s.step(1)
    pred = s.learn_predictions().astype(np.float64)
    Xn = ((F.T - shift.astype(np.float32)) * scale.astype(np.float32)).astype(np.float64)
    want = oracle.mlp_forward(P.astype(np.float64), Xn)
    assert np.abs(pred - want).max() <= 0.03 * max(1.0, np.abs(want).max())
    assert np.array_equal(s.learn_flags() != 0, pred < 0.0)


def test_tensor_core_gradient_matches_oracle():
    """BF16 tensor-core loss and gradient (forward, dL/dh1 = D2 W2 and the weight
    gradients as tcgen05 MMAs, FP32 accumulation): norm-wise within 1e-2 of the
    FP64 oracle gradient, loss within 1e-2."""
    rng = np.random.default_rng(27)
    P = (rng.standard_normal(dvm.MLP_NPARAM) * 0.3).astype(np.float32)
    X = rng.standard_normal((1000, 10)).astype(np.float32)
    y = rng.standard_normal(1000).astype(np.float32)
    m = dvm.Mlp(dvm.BF16S)
    m.set_params(P)
    loss, g = m.loss_grad(X, y)
    lo, go = oracle.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - lo) <= 1e-2 * lo, (loss, lo)
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    assert rel <= 1e-2, rel
    # every parameter block is there (no block left at zero)
    for a, b in ((0, 640), (640, 704), (704, 4800), (4800, 4864), (4864, 4928), (4928, 4929)):
        assert np.linalg.norm(g[a:b] - go[a:b]) <= 5e-2 * np.linalg.norm(go[a:b]) + 1e-6, (a, b)


def test_tensor_core_training_lowers_the_loss():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((20000, 10)).astype(np.float32)
    y = (np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.1 * X[:, 7]).astype(np.float32)
    P0 = (rng.standard_normal(dvm.MLP_NPARAM) * 0.1).astype(np.float32)
    m = dvm.Mlp(dvm.BF16S)
    m.set_params(P0)
    l0, _ = m.loss_grad(X, y)
    m.train(X, y, epochs=8, batch=512, lr=3e-3)
    l2, _ = m.loss_grad(X, y)
    assert l2 < 0.2 * l0, (l0, l2)
