"""Test-side helpers: conserved moments from primitive fields (Eqs. Mo and E of the
paper) and small utilities shared by the tests.  Not used by the library."""
import numpy as np

import oracle


def conserved(case) -> np.ndarray:
    """U = (rho, rho u, rho |u|^2 / 2 + d rho T / 2) per cell, SoA (d+2, Nc)."""
    d = case.d
    U = np.zeros((d + 2, case.ncells))
    U[0] = case.rho
    for i in range(d):
        U[1 + i] = case.rho * case.u[i]
    U[d + 1] = 0.5 * case.rho * (case.u ** 2).sum(0) + 0.5 * d * case.rho * case.T
    return U


def grid(case, scheme=None, subcycles=None) -> oracle.Grid:
    return oracle.Grid(d=case.d, nx=tuple(case.nx), dx=case.dx, nv=tuple(case.nv),
                       kmin=tuple(case.kmin), dv=case.dv, p=case.p, bc=tuple(case.bc),
                       scheme=case.scheme if scheme is None else scheme,
                       subcycles=case.subcycles if subcycles is None else subcycles)


def oracle_run(case, steps=None, scheme=None, subcycles=None, U0=None):
    g = grid(case, scheme, subcycles)
    s = oracle.Scheme(g, tau=case.tau)
    s.set_moments(conserved(case) if U0 is None else U0)
    s.step(case.steps if steps is None else steps)
    return s


def velocities(g: oracle.Grid) -> np.ndarray:
    """(3, Nv) velocity components, x index fastest."""
    ks = [np.arange(g.kmin[i], g.kmin[i] + g.nv[i]) if i < g.d else np.zeros(1)
          for i in range(3)]
    KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    return np.stack([KX.ravel(), KY.ravel(), KZ.ravel()]) * g.dv


def velocity_indices(g: oracle.Grid) -> np.ndarray:
    ks = [np.arange(g.kmin[i], g.kmin[i] + g.nv[i]) if i < g.d else np.zeros(1, dtype=int)
          for i in range(3)]
    KZ, KY, KX = np.meshgrid(ks[2], ks[1], ks[0], indexing="ij")
    return np.stack([KX.ravel(), KY.ravel(), KZ.ravel()]).astype(np.int64)


def paper_vortex_errors() -> dict:
    """{(scheme, norm): errors at the meshes 25, 50, 100, 200, 300, 400} from the
    isentropic-vortex table of Section 5.2 (tests/golden/vortex_errors.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "vortex_errors.txt")
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, norm, *vals = line.split()
            out[(getattr(oracle, name), norm)] = np.array([float(v) for v in vals])
    return out


VORTEX_MESHES = (25, 50, 100, 200, 300, 400)


def vortex_errors(case, rho) -> tuple:
    """The relative L1 and L-infinity density errors of Section 5.2 against the
    translated exact vortex."""
    ex = case.extra["rho_exact"]
    return (np.abs(rho - ex).sum() / np.abs(ex).sum(),
            np.abs(rho - ex).max() / np.abs(ex).max())
