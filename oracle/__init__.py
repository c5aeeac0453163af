"""Python access to the FP64 CPU oracle (``dvm_oracle.c``, ``riemann.c``, ``mlp.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library never
imports, links or calls it.  This module only marshals numpy arrays into the C
oracle; all arithmetic lives in the C sources, which follow the paper's Sections
3-4 step by step.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["dvm_oracle.c", "riemann.c", "mlp.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

FKS, HOFKS, HOFKS_UNLIMITED, HOFKS_WENO, FKS_STRANG = 0, 1, 2, 3, 4
PERIODIC, OUTFLOW = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no FMA contraction, so x86 and Arm agree)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "dvm_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-Wall", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(C.Structure):
    _fields_ = [("d", C.c_int), ("nx", C.c_int * 3), ("dx", C.c_double),
                ("bc", C.c_int * 3), ("nv", C.c_int * 3), ("kmin", C.c_int * 3),
                ("dv", C.c_double), ("p", C.c_int), ("scheme", C.c_int),
                ("subcycles", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        dp = C.POINTER(C.c_double)
        L.orc_offset.restype = C.c_longlong
        L.orc_offset.argtypes = [C.c_longlong] * 3
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(_Config), dp, C.c_double]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_moments.argtypes = [C.c_void_p, dp]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_get_moments.argtypes = [C.c_void_p, dp]
        L.orc_get_f.argtypes = [C.c_void_p, dp]
        L.orc_get_parts.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_info.argtypes = [C.c_void_p, dp, C.POINTER(C.c_longlong),
                               C.POINTER(C.c_int), dp]
        for name in ("orc_matrices",):
            getattr(L, name).argtypes = [C.POINTER(_Config), dp, dp]
        for name in ("orc_maxwellian", "orc_equilibrium"):
            getattr(L, name).argtypes = [C.POINTER(_Config), dp, dp]
        L.orc_project.argtypes = [C.POINTER(_Config), dp, dp, dp]
        L.orc_euler_flux.argtypes = [C.c_int, dp, C.c_int, dp]
        L.orc_euler_flux.restype = None
        L.orc_euler_alpha.argtypes = [C.POINTER(_Config), dp, dp]
        L.orc_muscl_step.argtypes = [C.POINTER(_Config), dp, C.c_double, dp,
                                     C.c_int, dp]
        L.orc_weno5_reconstruct.argtypes = [dp, C.c_int, C.c_int, dp]
        L.orc_weno_step.argtypes = [C.POINTER(_Config), dp, C.c_double, dp, C.c_int, dp]
        L.orc_riemann_exact.argtypes = [C.c_double] * 7 + [dp, C.c_int, dp, dp, dp, dp, dp]
        L.orc_step_flagged.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte), C.c_int]
        L.orc_set_lambda.argtypes = [C.c_void_p, dp]
        L.orc_set_lambda.restype = None
        L.orc_clone.restype = C.c_void_p
        L.orc_clone.argtypes = [C.c_void_p]
        L.orc_noneq.argtypes = [C.POINTER(_Config), dp, dp, dp]
        L.orc_features.argtypes = [C.POINTER(_Config), dp, dp, dp]
        L.orc_mlp_forward.argtypes = [C.c_int, dp, dp, dp]
        L.orc_mlp_loss_grad.restype = C.c_double
        L.orc_mlp_loss_grad.argtypes = [C.c_int, dp, dp, dp, dp]
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Grid:
    """Phase-space grid of the scheme (mirrors ``orc_config``)."""
    d: int
    nx: tuple
    dx: float
    nv: tuple
    kmin: tuple
    dv: float
    p: int = 1
    bc: tuple = (PERIODIC, PERIODIC, PERIODIC)
    scheme: int = HOFKS
    subcycles: int = 0

    def cstruct(self) -> _Config:
        c = _Config()
        c.d = self.d
        pad = lambda t, v: tuple(t) + (v,) * (3 - len(t))
        c.nx[:] = pad(self.nx, 1)
        c.dx = self.dx
        c.bc[:] = pad(self.bc, PERIODIC)
        c.nv[:] = pad(self.nv, 1)
        c.kmin[:] = pad(self.kmin, 0)
        c.dv = self.dv
        c.p = self.p
        c.scheme = self.scheme
        c.subcycles = self.subcycles
        return c

    @property
    def ncells(self) -> int:
        return int(np.prod(self.nx))

    @property
    def nvel(self) -> int:
        return int(np.prod(self.nv))

    @property
    def nmom(self) -> int:
        return self.d + 2

    @property
    def dt(self) -> float:
        return self.dx / (self.p * self.dv)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def offset(k: int, n: int, p: int) -> int:
    return int(lib().orc_offset(k, n, p))


def matrices(g: Grid):
    Cm = np.zeros((g.nmom, g.nvel))
    A = np.zeros((g.nmom, g.nmom))
    cfg = g.cstruct()
    _check(lib().orc_matrices(C.byref(cfg), _ptr(Cm), _ptr(A)), "matrices")
    return Cm, A


def maxwellian(g: Grid, U) -> np.ndarray:
    U = _f64(U)
    out = np.zeros(g.nvel)
    cfg = g.cstruct()
    _check(lib().orc_maxwellian(C.byref(cfg), _ptr(U), _ptr(out)), "maxwellian")
    return out


def equilibrium(g: Grid, U) -> np.ndarray:
    U = _f64(U)
    out = np.zeros(g.nvel)
    cfg = g.cstruct()
    _check(lib().orc_equilibrium(C.byref(cfg), _ptr(U), _ptr(out)), "equilibrium")
    return out


def project(g: Grid, ftilde, U) -> np.ndarray:
    ftilde, U = _f64(ftilde), _f64(U)
    out = np.zeros(g.nvel)
    cfg = g.cstruct()
    _check(lib().orc_project(C.byref(cfg), _ptr(ftilde), _ptr(U), _ptr(out)), "project")
    return out


def euler_flux(d: int, U, direction: int) -> np.ndarray:
    U = _f64(U)
    out = np.zeros(d + 2)
    lib().orc_euler_flux(d, _ptr(U), direction, _ptr(out))
    return out


def euler_alpha(g: Grid, U) -> np.ndarray:
    U = _f64(U)
    out = np.zeros(3)
    cfg = g.cstruct()
    _check(lib().orc_euler_alpha(C.byref(cfg), _ptr(U), _ptr(out)), "alpha")
    return out


def muscl_step(g: Grid, W, dt: float, alpha, limited: bool = True) -> np.ndarray:
    W = _f64(W)
    a = _f64(np.asarray(list(alpha) + [0.0] * (3 - len(alpha))))
    out = np.zeros_like(W)
    cfg = g.cstruct()
    _check(lib().orc_muscl_step(C.byref(cfg), _ptr(W), dt, _ptr(a), int(limited), _ptr(out)),
           "muscl")
    return out


def weno5_reconstruct(v, linear: bool = False) -> np.ndarray:
    """Left-biased WENO5 values at j+1/2 of the periodic samples v."""
    v = _f64(v)
    out = np.zeros_like(v)
    _check(lib().orc_weno5_reconstruct(_ptr(v), len(v), int(linear), _ptr(out)), "weno5")
    return out


def weno_step(g: Grid, W, dt: float, alpha, linear: bool = False) -> np.ndarray:
    W = _f64(W)
    a = _f64(np.asarray(list(alpha) + [0.0] * (3 - len(alpha))))
    out = np.zeros_like(W)
    cfg = g.cstruct()
    _check(lib().orc_weno_step(C.byref(cfg), _ptr(W), dt, _ptr(a), int(linear), _ptr(out)), "weno")
    return out


def riemann_exact(gamma, left, right, xi):
    """Exact Euler Riemann solution; left/right = (rho, u, p); returns rho, u, p, p*, u*."""
    xi = _f64(xi)
    n = xi.size
    r, u, p = np.zeros(n), np.zeros(n), np.zeros(n)
    ps, us = C.c_double(), C.c_double()
    _check(lib().orc_riemann_exact(gamma, *left, *right, _ptr(xi), n, _ptr(r), _ptr(u),
                                   _ptr(p), C.byref(ps), C.byref(us)), "riemann")
    return r, u, p, ps.value, us.value


@dataclass
class Scheme:
    """FKS/HOFKS state held by the oracle; f is kept at cell positions."""
    grid: Grid
    tau: object = np.inf
    _h: object = field(default=None, repr=False)

    def __post_init__(self):
        self._cfg = self.grid.cstruct()
        if np.isscalar(self.tau):
            h = lib().orc_create(C.byref(self._cfg), None, float(self.tau))
        else:
            self._tau_arr = _f64(self.tau)
            assert self._tau_arr.size == self.grid.ncells
            h = lib().orc_create(C.byref(self._cfg), _ptr(self._tau_arr), 0.0)
        if not h:
            raise RuntimeError("oracle create failed")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def set_moments(self, U):
        U = _f64(U).reshape(self.grid.nmom, self.grid.ncells)
        _check(lib().orc_set_moments(self._h, _ptr(U)), "set_moments")

    def step(self, n: int = 1):
        _check(lib().orc_step(self._h, int(n)), "step")

    def moments(self) -> np.ndarray:
        out = np.zeros((self.grid.nmom, self.grid.ncells))
        lib().orc_get_moments(self._h, _ptr(out))
        return out

    def f(self) -> np.ndarray:
        out = np.zeros((self.grid.nvel, self.grid.ncells))
        lib().orc_get_f(self._h, _ptr(out))
        return out

    def parts(self):
        shape = (self.grid.nmom, self.grid.ncells)
        UE, UM, Us = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        lib().orc_get_parts(self._h, _ptr(UE), _ptr(UM), _ptr(Us))
        return UE, UM, Us

    def step_flagged(self, flags, keep_raw: bool = False):
        """One HOFKS step with the flagged cells at equilibrium (lambda -> 0 form)."""
        fl = np.ascontiguousarray(np.asarray(flags) != 0, dtype=np.uint8)
        assert fl.size == self.grid.ncells
        _check(lib().orc_step_flagged(self._h, fl.ctypes.data_as(C.POINTER(C.c_ubyte)),
                                      int(keep_raw)), "step_flagged")

    def set_lambda(self, lam):
        """Replace the per-cell lambda (e.g. a flagged cell's lambda -> 0)."""
        self._lam = _f64(lam)
        assert self._lam.size == self.grid.ncells
        lib().orc_set_lambda(self._h, _ptr(self._lam))

    def clone(self) -> "Scheme":
        other = Scheme.__new__(Scheme)
        other.grid, other.tau = self.grid, self.tau
        other._cfg = self.grid.cstruct()
        other._h = lib().orc_clone(self._h)
        if not other._h:
            raise RuntimeError("oracle clone failed")
        return other

    def info(self):
        dt, n, m = C.c_double(), C.c_longlong(), C.c_int()
        alpha = np.zeros(3)
        lib().orc_info(self._h, C.byref(dt), C.byref(n), C.byref(m), _ptr(alpha))
        return {"dt": dt.value, "n": n.value, "m": m.value, "alpha": alpha}


def noneq(g: Grid, f, U) -> np.ndarray:
    """log10 of the discrete-L1 distance of f from E[U], relative to ||E[U]||, per cell."""
    f = _f64(f).reshape(g.nvel, g.ncells)
    U = _f64(U).reshape(g.nmom, g.ncells)
    out = np.zeros(g.ncells)
    cfg = g.cstruct()
    _check(lib().orc_noneq(C.byref(cfg), _ptr(f), _ptr(U), _ptr(out)), "noneq")
    return out


def features(g: Grid, U, tau) -> np.ndarray:
    """The ten regime features per cell, shape (10, Nc)."""
    U = _f64(U).reshape(g.nmom, g.ncells)
    tau = _f64(np.broadcast_to(np.asarray(tau, dtype=np.float64), (g.ncells,)))
    out = np.zeros((10, g.ncells))
    cfg = g.cstruct()
    _check(lib().orc_features(C.byref(cfg), _ptr(U), _ptr(tau), _ptr(out)), "features")
    return out


def mlp_forward(W, X) -> np.ndarray:
    """FP64 forward pass of the 10-64-64-1 tanh MLP; W is the packed parameter vector."""
    W, X = _f64(W), _f64(X)
    n = X.shape[0]
    out = np.zeros(n)
    lib().orc_mlp_forward(n, _ptr(W), _ptr(X), _ptr(out))
    return out


def mlp_loss_grad(W, X, y):
    """Mean-squared-error loss and its gradient with respect to the packed parameters."""
    W, X, y = _f64(W), _f64(X), _f64(y)
    g = np.zeros_like(W)
    loss = lib().orc_mlp_loss_grad(X.shape[0], _ptr(W), _ptr(X), _ptr(y), _ptr(g))
    return loss, g
