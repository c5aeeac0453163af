"""Pins of the oracle's learned-regime pieces: the flagged step, the regime
features and the non-equilibrium label.

A flagged cell is treated with the lambda -> 0 form of HOFKS (Theorem 1,
Section 4.3.1): its f^n is E[U^n] and its lambda is 0.  The pins tie that to
the plain scheme (which the other oracle pins fix), to conservation, to the
equilibrium identities, to a brute-force rebuild of one step and to closed
forms of central differences.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from tests.test_oracle_pins import centre_in_piece, kkt_project, piece_owner, rand_U, small_grid


def blocky_flags(rng, nx, frac=0.5, block=2):
    """Seeded flag mask made of block-wide tiles (regions, as a classifier gives)."""
    shape = tuple(reversed(nx))
    coarse = rng.uniform(size=tuple(-(-s // block) for s in shape)) < frac
    coarse.flat[0], coarse.flat[-1] = True, False  # always a mix
    fl = coarse
    for ax in range(len(shape)):
        fl = np.repeat(fl, block, axis=ax)
    fl = fl[tuple(slice(0, s) for s in shape)]
    return np.ascontiguousarray(fl.ravel().astype(np.uint8))


def stepped_scheme(g, tau, seed=3):
    rng = np.random.default_rng(seed)
    s = oracle.Scheme(g, tau=tau)
    s.set_moments(rand_U(rng, g.d, g.ncells))
    s.step(1)  # leave equilibrium first
    return s


@pytest.mark.parametrize("d", [1, 2])
def test_no_flags_is_the_plain_step(d):
    g = small_grid(d, n=6, nv=8)
    a = stepped_scheme(g, 1e-2)
    b = a.clone()
    a.step(1)
    b.step_flagged(np.zeros(g.ncells))
    assert np.array_equal(a.moments(), b.moments())
    assert np.array_equal(a.f(), b.f())


@pytest.mark.parametrize("d", [1, 2])
def test_flagged_step_is_the_plain_step_with_lambda_zero_there(d):
    """Flagging c equals the plain HOFKS step with lambda_c = 0: moments and raw
    f bit for bit; without keep_raw the flagged cells end at E[U^{n+1}]."""
    g = small_grid(d, n=6, nv=8)
    rng = np.random.default_rng(5)
    tau = rng.uniform(1e-3, 1e-1, g.ncells)
    fl = blocky_flags(rng, g.nx)
    assert 0 < fl.sum() < g.ncells
    a = stepped_scheme(g, tau)
    raw, kept, plain = a.clone(), a.clone(), a.clone()
    lam = np.exp(-g.dt / tau)
    plain.set_lambda(np.where(fl != 0, 0.0, lam))
    plain.step(1)
    raw.step_flagged(fl, keep_raw=True)
    kept.step_flagged(fl)
    assert np.array_equal(raw.moments(), plain.moments())
    assert np.array_equal(kept.moments(), plain.moments())
    assert np.array_equal(raw.f(), plain.f())
    for a_, b_ in zip(raw.parts(), plain.parts()):
        assert np.array_equal(a_, b_)
    f, U = kept.f(), kept.moments()
    Cm, _ = oracle.matrices(g)
    for c in np.flatnonzero(fl):
        E = oracle.equilibrium(g, U[:, c])
        assert np.abs(f[:, c] - E).max() <= 1e-15 * np.abs(E).max()
        np.testing.assert_allclose(Cm @ f[:, c], U[:, c], rtol=1e-13, atol=1e-14)
    keep = fl == 0
    assert np.array_equal(f[:, keep], plain.f()[:, keep])


def test_all_flagged_is_the_muscl_scheme():
    """Every cell flagged (uniform tau): U^{n+1} is the Euler MUSCL solution of U^n
    over dt (the lambda -> 0 limit of Theorem 1), whatever f^n was."""
    g = small_grid(1, n=16, nv=16, dv=0.5)
    a = stepped_scheme(g, 3e-2, seed=9)
    U0 = a.moments()
    a.step_flagged(np.ones(g.ncells))
    t, W = 0.0, U0.copy()
    while True:
        alpha = oracle.euler_alpha(g, W)
        dtE = 0.5 * g.dx / alpha[:1].sum()
        last = dtE >= g.dt - t
        dtE = g.dt - t if last else dtE
        W = oracle.muscl_step(g, W, dtE, alpha[:1])
        t += dtE
        if last:
            break
    np.testing.assert_allclose(a.moments(), W, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("d", [1, 2])
def test_flagged_periodic_runs_conserve(d):
    g = small_grid(d, n=8, nv=8)
    rng = np.random.default_rng(7)
    tau = 10.0 ** rng.uniform(-4, 0, g.ncells)
    s = stepped_scheme(g, tau, seed=11)
    U0 = s.moments()
    for _ in range(4):
        s.step_flagged(blocky_flags(rng, g.nx, 0.6))
    U = s.moments()
    assert np.all(np.abs(U.sum(1) - U0.sum(1)) <= 1e-13 * np.abs(U0).sum(1).max())


def test_uniform_equilibrium_is_a_fixed_point_with_flags():
    """All cells flagged: lambda_eff = 0 everywhere and a uniform equilibrium is a
    fixed point.  A partial mask makes lambda_eff jump between 0 and lambda, so
    W = (1 - lambda_eff) U is no longer uniform (as with any tau field): the state
    then moves by O(lambda) only."""
    g = small_grid(2, n=6, nv=10, dv=0.8)
    U0 = np.tile(np.array([[1.1], [0.2], [-0.1], [1.4]]), (1, g.ncells))
    for mask, tol in ((np.ones(g.ncells, dtype=np.uint8), 1e-14),
                      (blocky_flags(np.random.default_rng(2), g.nx), None)):
        s = oracle.Scheme(g, tau=1e-2)
        s.set_moments(U0)
        f0 = s.f()
        s.step_flagged(mask)
        lam = np.exp(-g.dt / 1e-2)
        bound = tol if tol is not None else 50 * lam
        assert np.abs(s.f() - f0).max() <= bound * np.abs(f0).max()
        assert np.abs(s.moments() - U0).max() <= bound * np.abs(U0).max()


def test_flags_on_free_cells_are_ignored():
    g = small_grid(1, n=6, nv=8)
    tau = np.full(g.ncells, 1e-2)
    tau[2] = np.inf
    a = stepped_scheme(g, tau)
    b = a.clone()
    fl = np.zeros(g.ncells, dtype=np.uint8)
    fl[2] = 1
    a.step(1)
    b.step_flagged(fl)
    assert np.array_equal(a.moments(), b.moments())
    assert np.array_equal(a.f(), b.f())


def test_flagged_step_brute_force_tiny_case():
    """5 cells x 4 velocities, p = 2: rebuild one flagged step from the definitions
    (piece geometry in exact rationals, projections as KKT solves, U_E from the
    oracle's MUSCL of W = (1 - lambda_eff) U^n) and compare f and U."""
    g = oracle.Grid(d=1, nx=(5,), dx=0.2, nv=(4,), kmin=(-2,), dv=1.1, p=2,
                    bc=(oracle.PERIODIC,), scheme=oracle.HOFKS)
    rng = np.random.default_rng(12)
    tau = rng.uniform(0.05, 0.5, 5)
    s = oracle.Scheme(g, tau=tau)
    s.set_moments(rand_U(rng, 1, 5))
    s.step(1)
    f, U = s.f(), s.moments()
    fl = np.array([1, 0, 0, 1, 1], dtype=np.uint8)
    s.step_flagged(fl)
    n = 1
    Cm, _ = oracle.matrices(g)
    lam = np.where(fl != 0, 0.0, np.exp(-g.dt / tau))
    Eq = np.stack([kkt_project(Cm, oracle.maxwellian(g, U[:, c]), U[:, c]) for c in range(5)], 1)
    f = np.where(fl[None, :] != 0, Eq, f)
    kv = np.arange(-2, 2)
    UE, _, _ = s.parts()
    fnew = np.zeros_like(f)
    for c in range(5):
        for k in range(4):
            j = piece_owner(c, Fraction(int(kv[k]) * (n + 1), 2))
            sc = centre_in_piece(j, Fraction(int(kv[k]) * n, 2)) % 5
            fnew[k, c] = lam[sc] * f[k, sc]
        b = np.array([(1 - lam[sc]) * Eq[k, sc] for k, sc in
                      ((k, centre_in_piece(piece_owner(c, Fraction(int(kv[k]) * (n + 1), 2)),
                                           Fraction(int(kv[k]) * n, 2)) % 5) for k in range(4))])
        fnew[:, c] += kkt_project(Cm, b, UE[:, c])
    Unew = Cm @ fnew
    for c in np.flatnonzero(fl):
        fnew[:, c] = kkt_project(Cm, oracle.maxwellian(g, Unew[:, c]), Unew[:, c])
    np.testing.assert_allclose(s.f(), fnew, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s.moments(), Unew, rtol=1e-12, atol=1e-14)
    # U_E is the MUSCL solution from W = (1 - lambda_eff) U^n
    W = (1 - lam) * U
    t = 0.0
    while True:
        alpha = oracle.euler_alpha(g, W)
        dtE = 0.5 * g.dx / alpha[0]
        last = dtE >= g.dt - t
        dtE = g.dt - t if last else dtE
        W = oracle.muscl_step(g, W, dtE, alpha[:1])
        t += dtE
        if last:
            break
    np.testing.assert_allclose(UE, W, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------- label


def test_noneq_of_an_equilibrium_is_the_floor_and_scales_exactly():
    g = small_grid(2, n=4, nv=10, dv=0.8)
    U = rand_U(np.random.default_rng(4), 2, g.ncells)
    E = np.stack([oracle.equilibrium(g, U[:, c]) for c in range(g.ncells)], 1)
    assert np.all(oracle.noneq(g, E, U) == -12.0)
    # f = (1 + s) E: ||f - E||_1 / ||E||_1 = |s| exactly
    s = np.array([1e-3, -2e-2, 0.25, -0.5] * 4)
    got = oracle.noneq(g, E * (1 + s), U)
    np.testing.assert_allclose(got, np.log10(np.abs(s)), rtol=0, atol=1e-12)
    # mixed signs in the perturbation: the L1 norm, not the L2 norm
    pert = np.where(np.arange(g.nvel)[:, None] % 2 == 0, 1.0, -1.0) * 1e-3 * np.abs(E)
    got = oracle.noneq(g, E + pert, U)
    np.testing.assert_allclose(got, np.log10(1e-3), atol=1e-12)


# ---------------------------------------------------------------------- features


def sine_state(n, a=0.3, b=0.2, cy=0.1, T=lambda X, Y: 1.0 + 0 * X):
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = np.exp(a * np.sin(2 * np.pi * X))
    ux = b * np.sin(2 * np.pi * Y)
    uy = cy * np.sin(2 * np.pi * X)
    th = T(X, Y)
    U = np.stack([rho, rho * ux, rho * uy, 0.5 * rho * (ux ** 2 + uy ** 2) + rho * th])
    return X, Y, U.reshape(4, -1), rho, ux, uy, th


def test_features_match_the_central_difference_closed_forms():
    """Central differences of sin(2 pi x) are exactly cos(2 pi x) sin(2 pi dx)/dx,
    so every gradient feature has a closed form on sine fields."""
    n = 16
    g = oracle.Grid(d=2, nx=(n, n), dx=1.0 / n, nv=(8, 8), kmin=(-4, -4), dv=1.0)
    X, Y, U, rho, ux, uy, th = sine_state(n, T=lambda X, Y: np.exp(0.4 * np.sin(2 * np.pi * Y)))
    tau = 10.0 ** np.linspace(-5, -1, n * n)
    F = oracle.features(g, U, tau)
    k = np.sin(2 * np.pi / n) * n  # d/dx of sin(2 pi x), discretely, per unit cos
    cx, cy_ = np.cos(2 * np.pi * X).ravel(), np.cos(2 * np.pi * Y).ravel()
    np.testing.assert_allclose(F[0], rho.ravel(), rtol=1e-14)
    np.testing.assert_allclose(F[1], ux.ravel(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(F[2], uy.ravel(), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(F[3], th.ravel(), rtol=1e-13)
    np.testing.assert_allclose(F[4], np.log10(tau), rtol=1e-14)
    sq = np.sqrt(th.ravel())
    K = np.stack([tau * sq * np.abs(0.3 * k * cx),       # grad ln rho = (0.3 k cos x, 0)
                  tau * sq * np.abs(0.4 * k * cy_),      # grad ln theta = (0, 0.4 k cos y)
                  tau * 0.0,                             # div u = d_x ux + d_y uy = 0
                  tau * np.abs(0.2 * k * cy_),           # d_y ux
                  tau * np.abs(0.1 * k * cx)])           # d_x uy
    want = np.log10(np.maximum(K, 1e-12))
    np.testing.assert_allclose(F[5:], want, rtol=0, atol=1e-10)


def test_feature_divergence_and_uniform_state():
    n = 12
    g = oracle.Grid(d=2, nx=(n, n), dx=1.0 / n, nv=(8, 8), kmin=(-4, -4), dv=1.0)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux, uy = 0.2 * np.sin(2 * np.pi * X), 0.3 * np.sin(2 * np.pi * Y)
    U = np.stack([np.ones_like(X), ux, uy, 0.5 * (ux ** 2 + uy ** 2) + 1.0]).reshape(4, -1)
    F = oracle.features(g, U, 1e-2)
    k = np.sin(2 * np.pi / n) * n
    div = 0.2 * k * np.cos(2 * np.pi * X) + 0.3 * k * np.cos(2 * np.pi * Y)
    np.testing.assert_allclose(F[7], np.log10(np.maximum(1e-2 * np.abs(div.ravel()), 1e-12)),
                               atol=1e-9)
    U1 = np.tile(np.array([[0.7], [0.1], [0.0], [1.0]]), (1, n * n))
    F1 = oracle.features(g, U1, 3e-3)
    assert np.all(F1[5:] == -12.0)
    np.testing.assert_allclose(F1[3], (2 * 1.0 / 0.7 - (0.1 / 0.7) ** 2) / 2, rtol=1e-15)
