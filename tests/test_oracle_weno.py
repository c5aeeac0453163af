"""Pins of the oracle's WENO Euler solver (Section 4.3.3 names WENO as a higher-order
alternative to MUSCL inside HOFKS; the oracle takes finite-difference WENO5 of Jiang
and Shu on Lax-Friedrichs split fluxes, SSP Runge-Kutta 3 per Euler sub-step).

Each pin is a fact fixed by the mathematics, not a retyped formula:
* every candidate stencil is exact on quadratics, whatever the weights (the
  reconstruction of the primitive's interface value from point samples);
* with the optimal linear weights the flux difference is the exact derivative of any
  quartic (fifth order), and the error falls at rate 5 on smooth data;
* the nonlinear weights converge on smooth data and do not overshoot a step, where
  the linear weights do;
* the scheme conserves periodic totals, keeps uniform states, is mirror symmetric,
  and at tau = 0 HOFKS-WENO is the WENO Euler scheme sub-stepped over dt;
* on the smooth entropy wave in the fluid limit its error falls at rate ~5 (MUSCL:
  2), and on the Sod tube it is closer to the exact Riemann solution than MUSCL.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved, grid, oracle_run


def poly(coef, x):
    return sum(c * x ** k for k, c in enumerate(coef))


@pytest.mark.parametrize("linear", [False, True])
def test_candidate_stencils_are_exact_on_quadratics(linear):
    """f = a + b x + c x^2 sampled at x_j = j is the cell average of
    h = f - c/12; every candidate (and so any convex blend) returns h(j + 1/2)."""
    j = np.arange(24, dtype=float)
    a, b, c = 0.3, -1.1, 0.7
    r = oracle.weno5_reconstruct(poly((a, b, c), j), linear)
    exact = poly((a, b, c), j + 0.5) - c / 12.0
    inner = slice(3, -3)  # stencils that do not wrap around the periodic array
    assert np.abs(r[inner] - exact[inner]).max() <= 1e-13 * np.abs(exact).max()


def test_linear_weights_differentiate_quartics_exactly():
    """Fifth order: (h_{j+1/2} - h_{j-1/2}) equals f'(x_j) for every quartic f."""
    j = np.arange(24, dtype=float)
    q = (0.2, -0.5, 0.3, 0.05, -0.01)
    r = oracle.weno5_reconstruct(poly(q, j), linear=True)
    dq = tuple(k * q[k] for k in range(1, 5))
    d = r[4:-3] - r[3:-4]
    assert np.abs(d - poly(dq, j[4:-3])).max() <= 1e-12 * np.abs(poly(dq, j)).max()


def smooth_rates(linear):
    errs = []
    for n in (16, 32, 64, 128):
        x = np.arange(n) / n
        v = np.sin(2 * np.pi * x) + 0.5 * np.cos(4 * np.pi * x)
        r = oracle.weno5_reconstruct(v, linear)
        d = (r - np.roll(r, 1)) * n
        exact = 2 * np.pi * np.cos(2 * np.pi * x) - 2 * np.pi * np.sin(4 * np.pi * x)
        errs.append(np.abs(d - exact).max())
    return np.array(errs), np.log2(np.array(errs[:-1]) / np.array(errs[1:]))


def test_smooth_data_convergence_rates():
    errs, rates = smooth_rates(True)
    assert np.all(rates > 4.8), rates        # the optimal weights: fifth order
    errs_nl, rates_nl = smooth_rates(False)
    # the nonlinear weights tend to the optimal ones (slower at the critical points)
    assert np.all(rates_nl > 3.3), rates_nl
    assert errs_nl[-1] < 5e-5 * 2 * np.pi * 1.5  # relative to the largest |f'|


def test_nonlinear_weights_do_not_overshoot_a_step():
    v = np.where(np.arange(40) < 20, 0.0, 1.0)
    over = lambda r: max(r.max() - 1.0, -r.min())
    assert over(oracle.weno5_reconstruct(v, False)) < 1e-10
    assert over(oracle.weno5_reconstruct(v, True)) > 0.1  # unlimited high order rings


def weno_grid(nx=48, bc=oracle.PERIODIC):
    return oracle.Grid(d=1, nx=(nx,), dx=1.0 / nx, nv=(16,), kmin=(-8,), dv=0.5, p=1,
                       bc=(bc,), scheme=oracle.HOFKS_WENO)


def riemann_state(nx, left, right):
    x = (np.arange(nx) + 0.5) / nx
    rho = np.where(x < 0.5, left[0], right[0])
    u = np.where(x < 0.5, left[1], right[1])
    p = np.where(x < 0.5, left[2], right[2])
    return np.stack([rho, rho * u, p + 0.5 * rho * u * u])  # gamma = 3 in 1D: E = p + rho u^2/2


def test_weno_step_conserves_keeps_uniform_states_and_is_mirror_symmetric():
    g = weno_grid()
    W0 = riemann_state(48, (1.0, 0.3, 1.0), (0.3, -0.2, 0.4))
    alpha = oracle.euler_alpha(g, W0)
    W1 = oracle.weno_step(g, W0, 2e-3, alpha)
    assert np.all(np.abs(W1.sum(1) - W0.sum(1)) <= 1e-13 * np.abs(W0).sum(1))
    U = np.tile([[1.3], [0.4], [2.1]], (1, 48))
    assert np.abs(oracle.weno_step(g, U, 2e-3, alpha) - U).max() <= 1e-14 * 2.1
    # mirror x -> -x: density and energy mirrored, momentum mirrored and negated
    M = W0[:, ::-1].copy()
    M[1] = -M[1]
    M1 = oracle.weno_step(g, M, 2e-3, alpha)
    back = M1[:, ::-1].copy()
    back[1] = -back[1]
    assert np.abs(back - W1).max() <= 1e-13 * np.abs(W1).max()


def test_tau_zero_hofks_weno_is_the_weno_scheme():
    """lambda = 0: U^{n+1} = U_E, the WENO Euler scheme sub-stepped over dt."""
    case = W.entropy_wave_1d(40, tau=0.0)
    g = grid(case, scheme=oracle.HOFKS_WENO, subcycles=4)
    s = oracle.Scheme(g, tau=0.0)
    U0 = conserved(case)
    s.set_moments(U0)
    s.step(1)
    Wk = U0.copy()
    for _ in range(4):
        Wk = oracle.weno_step(g, Wk, case.dt / 4, oracle.euler_alpha(g, Wk))
    assert np.abs(s.moments() - Wk).max() <= 1e-14 * np.abs(Wk).max()


def test_periodic_hofks_weno_conserves():
    for tau in (1e-4, 1e-2):
        case = W.entropy_wave_1d(60, tau=tau)
        s = oracle_run(case, steps=5, scheme=oracle.HOFKS_WENO)
        U0, U = conserved(case), s.moments()
        scale = np.abs(U0).sum(1)
        scale[1] = scale[0]
        assert np.all(np.abs(U.sum(1) - U0.sum(1)) <= 1e-13 * scale)


def test_weno_has_higher_order_than_muscl_on_the_smooth_wave():
    """Fluid limit, dt_E ~ dx^2 (the time error out of the way): HOFKS-WENO falls at
    rate ~5, HOFKS-MUSCL at ~2, and WENO is the more accurate on every mesh."""
    errs = {}
    for scheme in (oracle.HOFKS, oracle.HOFKS_WENO):
        e = []
        for nx in (20, 40, 80):
            case = W.entropy_wave_1d(nx, tau=0.0)
            s = oracle_run(case, scheme=scheme, subcycles=nx // 2)
            x = (np.arange(nx) + 0.5) / nx
            exact = 1 + 0.2 * np.sin(2 * np.pi * (x - 0.5 * case.extra["t_final"]))
            e.append(np.abs(s.moments()[0] - exact).sum() / np.abs(exact).sum())
        errs[scheme] = np.array(e)
    rw = np.log2(errs[oracle.HOFKS_WENO][:-1] / errs[oracle.HOFKS_WENO][1:])
    rm = np.log2(errs[oracle.HOFKS][:-1] / errs[oracle.HOFKS][1:])
    assert np.all(rw > 4.5), rw
    assert np.all(rm < 2.3), rm
    assert np.all(errs[oracle.HOFKS_WENO] < errs[oracle.HOFKS])


def test_weno_sod_is_closer_to_the_exact_solution_than_muscl():
    for nx in (100, 200):
        e = {}
        for scheme in (oracle.HOFKS, oracle.HOFKS_WENO):
            case = W.sod_1d(nx=nx, tau=1e-4)
            s = oracle_run(case, scheme=scheme)
            t = case.steps * case.dt
            x = (np.arange(nx) + 0.5) / nx
            r, *_ = oracle.riemann_exact(3.0, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / t)
            e[scheme] = np.abs(s.moments()[0] - r).mean()
        assert e[oracle.HOFKS_WENO] < e[oracle.HOFKS], (nx, e)
