"""Pins of the oracle's Strang-split FKS (Section 4.2 names Strang splitting as the
more accurate alternative to its first-order splitting): every step is a relaxation
over dt/2, the exact transport over dt and a relaxation over dt/2.

A relaxation R_h keeps the moments of every cell and so its equilibrium E[U]; two of
them make a full one (R_h R_h = R, since lambda_h^2 = lambda), and E is its fixed
point.  From equilibrium initial data, Strang's state after n steps is therefore
R_h T (R T)^(n-1) f^0 while first-order FKS has R T (R T)^(n-1) f^0: the same
moments at every step, and f_S - E = (f_L - E) / lambda_h cell by cell.  These
facts, conservation and the limits tau = inf and tau = 0 pin the implementation.
"""
import numpy as np
import pytest

import oracle
from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved, grid


def cases():
    shear = W.shear_layer_2d(n=14, nv=10, steps=3, dv=1.0)     # a tau field
    return [W.sod_1d(nx=60, nv=24, tau=3e-3, dv=0.6),            # outflow
            W.quadrant_2d(n=12, nv=10, tau=2e-2, steps=3, dv=0.9),
            shear]


def equilibria(g, U):
    """E[U] of every cell, (N_v, N_c) (Eq. minimMax, cell by cell)."""
    return np.stack([oracle.equilibrium(g, U[:, c]) for c in range(U.shape[1])], axis=1)


def pair(case, steps):
    out = []
    for scheme in (oracle.FKS_STRANG, oracle.FKS):
        s = oracle.Scheme(grid(case, scheme), tau=case.tau)
        s.set_moments(conserved(case))
        out.append(s)
    return out


@pytest.mark.parametrize("case", cases(), ids=["sod_outflow", "quadrant", "shear_taufield"])
def test_strang_moments_equal_the_first_order_ones_at_every_step(case):
    st, lie = pair(case, 4)
    for _ in range(4):
        st.step(1)
        lie.step(1)
        U, V = st.moments(), lie.moments()
        assert np.abs(U - V).max() <= 1e-13 * np.abs(V).max()


@pytest.mark.parametrize("case", cases(), ids=["sod_outflow", "quadrant", "shear_taufield"])
def test_strang_f_is_the_half_relaxed_transported_state(case):
    """f_L - E = lambda_h (f_S - E): the first-order state is one more half
    relaxation of Strang's."""
    st, lie = pair(case, 3)
    st.step(3)
    lie.step(3)
    g = grid(case, oracle.FKS)
    E = equilibria(g, lie.moments())
    tau = np.broadcast_to(np.asarray(case.tau, dtype=float), (case.ncells,))
    lamh = np.exp(-g.dt / (2.0 * tau))
    fs, fl = st.f(), lie.f()
    assert np.abs((fl - E) - lamh * (fs - E)).max() <= 1e-13 * np.abs(fl).max()
    assert np.abs(fs - fl).max() > 1e-6 * np.abs(fl).max()  # and the two differ


def test_strang_free_transport_and_fluid_limit():
    case = W.quadrant_2d(n=11, nv=8, tau=np.inf, steps=3, dv=1.0)
    st, lie = pair(case, 3)
    st.step(3)
    lie.step(3)
    assert np.array_equal(st.f(), lie.f())  # lambda_h = 1: pure exact transport
    case0 = W.sod_1d(nx=40, nv=16, tau=0.0, dv=0.8)
    s = oracle.Scheme(grid(case0, oracle.FKS_STRANG), tau=0.0)
    s.set_moments(conserved(case0))
    s.step(2)
    E = equilibria(grid(case0, oracle.FKS), s.moments())
    assert np.abs(s.f() - E).max() <= 1e-14 * np.abs(E).max()


def test_strang_periodic_runs_conserve():
    case = W.quadrant_2d(n=12, nv=10, tau=5e-3, steps=3, dv=0.9)
    s = oracle.Scheme(grid(case, oracle.FKS_STRANG), tau=case.tau)
    U0 = conserved(case)
    s.set_moments(U0)
    s.step(5)
    scale = np.abs(U0).sum(1)
    scale[1:3] = scale[0]
    assert np.all(np.abs(s.moments().sum(1) - U0.sum(1)) <= 1e-13 * scale)
