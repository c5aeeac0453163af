"""ctypes binding of libdvm (include/dvm.h): argument marshalling only.

Every step of the scheme runs in the CUDA library; this module converts Python
values into the C structs and pointers of the ABI.  PyTorch supplies the device
workspace (its caching allocator) and the CUDA stream.  There is no CPU
fallback: if ``libdvm.so`` is missing or no GPU is visible, creating a solver
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdvm.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_STATE, ERR_CFL = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
ERR_TOO_LARGE = -9
PERIODIC, OUTFLOW = 0, 1
FKS, HOFKS, HOFKS_UNLIMITED, HOFKS_WENO, FKS_STRANG = 0, 1, 2, 3, 4
F64, F32, BF16S = 0, 1, 2
SELFTEST_GRID_BARRIER, SELFTEST_MBARRIER = 0, 1

# every symbol include/dvm.h declares (checked by the CPU tests)
EXPORTS = [
    "dvm_workspace_bytes", "dvm_create", "dvm_destroy", "dvm_set_stream", "dvm_last_error",
    "dvm_set_state_moments", "dvm_set_state_primitive", "dvm_step", "dvm_step_async",
    "dvm_sync_status", "dvm_moments", "dvm_moments_async", "dvm_moments_wait", "dvm_get_f", "dvm_last_parts", "dvm_info", "dvm_offsets",
    "dvm_save", "dvm_load", "dvm_launches_per_step", "dvm_kinetic_kernel", "dvm_kinetic_splits", "dvm_plan", "dvm_profile_begin",
    "dvm_profile_end",
    "dvm_equilibrium_noalloc", "dvm_selftest_timeout",
    "dvm_batch_create", "dvm_batch_destroy", "dvm_batch_last_error", "dvm_batch_sizes",
    "dvm_batch_moment_rows",
    "dvm_batch_set_state_moments", "dvm_batch_step", "dvm_batch_step_async",
    "dvm_batch_sync_status", "dvm_batch_moments", "dvm_batch_moments_async", "dvm_batch_moments_wait", "dvm_batch_get_f", "dvm_batch_info",
    "dvm_batch_set_tiling", "dvm_batch_autotune", "dvm_batch_kinetic_ms",
    "dvm_learn_enable", "dvm_learn_set_params", "dvm_learn_set_flags", "dvm_learn_flags",
    "dvm_learn_predictions", "dvm_learn_get_stats", "dvm_learn_step_checked", "dvm_features",
    "dvm_noneq",
    "dvm_mlp_create", "dvm_mlp_destroy", "dvm_mlp_set_params", "dvm_mlp_get_params",
    "dvm_mlp_forward", "dvm_mlp_loss_grad", "dvm_mlp_train",
]

NFEAT, MLP_HIDDEN = 10, 64
MLP_NPARAM = 64 * 10 + 64 + 64 * 64 + 64 + 64 + 1
LEARN_OFF, LEARN_GIVEN, LEARN_MLP = 0, 1, 2


class DvmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdvm status {code}: {msg}")
        self.code = code


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int * 3), ("x0", C.c_double * 3), ("dx", C.c_double)]


class _VSet(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("kmin", C.c_int * 3), ("dv", C.c_double),
                ("shift_den", C.c_int)]


class _Config(C.Structure):
    _fields_ = [("grid", _Grid), ("vel", _VSet), ("tau", C.c_double),
                ("tau_field", C.POINTER(C.c_double)), ("bc", (C.c_int * 2) * 3),
                ("scheme", C.c_int), ("precision", C.c_int), ("euler_subcycles", C.c_int),
                ("max_subcycles", C.c_int)]


class _LearnConfig(C.Structure):
    _fields_ = [("mode", C.c_int), ("mlp_precision", C.c_int), ("thr", C.c_float),
                ("check_every", C.c_int), ("check_samples", C.c_int), ("veto_radius", C.c_int),
                ("seed", C.c_ulonglong), ("feat_shift", C.c_float * NFEAT),
                ("feat_scale", C.c_float * NFEAT)]


class _LearnStats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("flagged", C.c_longlong),
                ("flagged_total", C.c_longlong), ("materialised", C.c_longlong),
                ("checks", C.c_longlong), ("checked", C.c_longlong), ("failed", C.c_longlong),
                ("vetoed", C.c_longlong), ("sum_abs_err", C.c_double),
                ("max_abs_err", C.c_double), ("max_true", C.c_double)]


class _TrainConfig(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_ulonglong)]


_lib = None


def lib():
    """Load libdvm.so (built by ``paper_1212_0204_gb300.build``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
        L.dvm_workspace_bytes.argtypes = [C.POINTER(_Config), C.POINTER(C.c_size_t)]
        L.dvm_create.argtypes = [C.POINTER(_Config), vp, vp, C.POINTER(vp)]
        L.dvm_destroy.argtypes = [vp]
        L.dvm_destroy.restype = None
        L.dvm_set_stream.argtypes = [vp, vp]
        L.dvm_last_error.argtypes = [vp]
        L.dvm_last_error.restype = C.c_char_p
        L.dvm_set_state_moments.argtypes = [vp, vp, ip]
        L.dvm_set_state_primitive.argtypes = [vp, vp, vp, vp, ip]
        L.dvm_step.argtypes = [vp, ip]
        L.dvm_step_async.argtypes = [vp, ip]
        L.dvm_sync_status.argtypes = [vp]
        L.dvm_moments.argtypes = [vp, vp, ip]
        L.dvm_moments_async.argtypes = [vp, vp, ip, C.POINTER(C.c_longlong)]
        L.dvm_moments_wait.argtypes = [vp, C.c_longlong]
        L.dvm_batch_moments_async.argtypes = [vp, vp, ip, C.POINTER(C.c_longlong)]
        L.dvm_batch_moments_wait.argtypes = [vp, C.c_longlong]
        L.dvm_get_f.argtypes = [vp, vp, ip]
        L.dvm_last_parts.argtypes = [vp, vp, vp, vp]
        L.dvm_info.argtypes = [vp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_int), dp]
        L.dvm_offsets.argtypes = [vp, C.c_longlong, C.POINTER(C.c_longlong)]
        L.dvm_save.argtypes = [vp, vp, C.POINTER(C.c_size_t)]
        L.dvm_load.argtypes = [vp, vp, C.c_size_t]
        L.dvm_launches_per_step.argtypes = [vp, C.POINTER(C.c_int)]
        L.dvm_kinetic_kernel.argtypes = [vp, C.POINTER(C.c_int)]
        L.dvm_kinetic_splits.argtypes = [vp, C.POINTER(C.c_int)]
        L.dvm_plan.argtypes = [C.POINTER(_Config), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.dvm_profile_begin.argtypes = [vp]
        L.dvm_profile_end.argtypes = [vp, dp, C.POINTER(C.c_int)]
        L.dvm_equilibrium_noalloc.argtypes = [C.POINTER(_Config), vp, vp, vp]
        L.dvm_selftest_timeout.argtypes = [C.c_int, vp, C.POINTER(C.c_int)]
        L.dvm_batch_create.argtypes = [C.POINTER(_Config), ip, vp, C.POINTER(vp)]
        L.dvm_batch_destroy.argtypes = [vp]
        L.dvm_batch_destroy.restype = None
        L.dvm_batch_last_error.argtypes = [vp]
        L.dvm_batch_last_error.restype = C.c_char_p
        L.dvm_batch_sizes.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
        L.dvm_batch_set_state_moments.argtypes = [vp, vp, ip]
        L.dvm_batch_step.argtypes = [vp, ip]
        L.dvm_batch_step_async.argtypes = [vp, ip]
        L.dvm_batch_sync_status.argtypes = [vp]
        L.dvm_batch_moments.argtypes = [vp, vp, ip]
        L.dvm_batch_get_f.argtypes = [vp, ip, vp]
        L.dvm_batch_info.argtypes = [vp, C.POINTER(C.c_longlong), vp, vp]
        L.dvm_batch_moment_rows.argtypes = [vp, C.POINTER(C.c_int)]
        L.dvm_batch_set_tiling.argtypes = [vp, ip, ip, ip, ip]
        L.dvm_batch_autotune.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(C.c_int), dp]
        L.dvm_batch_kinetic_ms.argtypes = [vp, ip, dp]
        L.dvm_learn_enable.argtypes = [vp, C.POINTER(_LearnConfig)]
        L.dvm_learn_set_params.argtypes = [vp, vp]
        L.dvm_learn_set_flags.argtypes = [vp, vp]
        L.dvm_learn_flags.argtypes = [vp, vp]
        L.dvm_learn_predictions.argtypes = [vp, vp]
        L.dvm_learn_get_stats.argtypes = [vp, C.POINTER(_LearnStats)]
        L.dvm_learn_step_checked.argtypes = [vp, ip, vp, vp]
        L.dvm_features.argtypes = [vp, vp]
        L.dvm_noneq.argtypes = [vp, vp]
        L.dvm_mlp_create.argtypes = [ip, vp, C.POINTER(vp)]
        L.dvm_mlp_destroy.argtypes = [vp]
        L.dvm_mlp_destroy.restype = None
        L.dvm_mlp_set_params.argtypes = [vp, vp]
        L.dvm_mlp_get_params.argtypes = [vp, vp]
        L.dvm_mlp_forward.argtypes = [vp, C.c_longlong, vp, vp]
        L.dvm_mlp_loss_grad.argtypes = [vp, C.c_longlong, vp, vp, vp, dp]
        L.dvm_mlp_train.argtypes = [vp, C.c_longlong, vp, vp, C.POINTER(_TrainConfig), dp]
        _lib = L
    return _lib


def make_config(d, nx, dx, nv, kmin, dv, p=1, bc=None, tau=float("inf"), tau_field=None,
                scheme=HOFKS, precision=F64, subcycles=0, max_subcycles=0, x0=None):
    """Fill the C ``dvm_config``; returns (struct, keep-alive list)."""
    pad = lambda t, v: list(t) + [v] * (3 - len(t))
    cfg = _Config()
    cfg.grid.dim = d
    cfg.grid.nx[:] = pad(nx, 1)
    cfg.grid.x0[:] = pad(x0 or (), 0.0)
    cfg.grid.dx = dx
    cfg.vel.n[:] = pad(nv, 1)
    cfg.vel.kmin[:] = pad(kmin, 0)
    cfg.vel.dv = dv
    cfg.vel.shift_den = p
    keep = []
    if tau_field is not None:
        arr = np.ascontiguousarray(tau_field, dtype=np.float64)
        keep.append(arr)
        cfg.tau_field = arr.ctypes.data_as(C.POINTER(C.c_double))
        cfg.tau = 0.0
    else:
        cfg.tau = tau
    bcs = pad(bc or (), PERIODIC)
    for i in range(3):
        cfg.bc[i][0] = bcs[i]
        cfg.bc[i][1] = bcs[i]
    cfg.scheme = scheme
    cfg.precision = precision
    cfg.euler_subcycles = subcycles
    cfg.max_subcycles = max_subcycles
    return cfg, keep


def config_from_case(case, precision=F64, scheme=None, subcycles=None):
    tau = case.tau
    field = None if np.isscalar(tau) else tau
    return make_config(case.d, case.nx, case.dx, case.nv, case.kmin, case.dv, case.p, case.bc,
                       tau=float(tau) if field is None else 0.0, tau_field=field,
                       scheme=case.scheme if scheme is None else scheme, precision=precision,
                       subcycles=case.subcycles if subcycles is None else subcycles)


def equilibrium_noalloc(cfg, U, f, stream=None) -> int:
    """f = E[U] through the allocation-free entry point; U and f are CUDA tensors
    (FP64, contiguous).  Returns the status code (0 on success)."""
    import torch
    assert U.is_cuda and f.is_cuda and U.dtype == torch.float64 and f.dtype == torch.float64
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib().dvm_equilibrium_noalloc(C.byref(cfg), C.c_void_p(U.data_ptr()),
                                         C.c_void_p(f.data_ptr()), C.c_void_p(s.cuda_stream))


def selftest_timeout(which: int, stream=None) -> int:
    """Run one of the library's bounded device waits on an event that never
    comes (dvm_selftest_timeout); returns the device status word it left
    (ERR_TIMEOUT when the wait gave up as designed)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libdvm needs a CUDA GPU; no CPU fallback exists")
    st = C.c_int(0)
    rc = lib().dvm_selftest_timeout(int(which), C.c_void_p(stream), C.byref(st))
    if rc:
        raise DvmError(rc, "selftest launch failed")
    return st.value


def plan(cfg) -> tuple:
    """(kinetic-pass kernel "window"/"generic", velocity splits) that dvm_create would
    choose for cfg; host only (no GPU needed)."""
    kind, splits = C.c_int(), C.c_int()
    rc = lib().dvm_plan(C.byref(cfg), C.byref(kind), C.byref(splits))
    if rc:
        raise DvmError(rc, "invalid configuration")
    return ("generic", "window")[kind.value], splits.value


def workspace_bytes(cfg) -> int:
    n = C.c_size_t()
    rc = lib().dvm_workspace_bytes(C.byref(cfg), C.byref(n))
    if rc:
        raise DvmError(rc, "invalid configuration")
    return n.value


class Solver:
    """One libdvm handle.  Device memory comes from a torch uint8 tensor and work
    runs on torch's current CUDA stream (or the one given)."""

    def __init__(self, cfg, keep=(), stream=None, torch_workspace=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libdvm needs a CUDA GPU; no CPU fallback exists")
        self._torch = torch
        self.cfg = cfg
        self._keep = list(keep)
        self.d = cfg.grid.dim
        self.nm = self.d + 2
        self.nc = int(np.prod([cfg.grid.nx[i] for i in range(3)]))
        self.nvel = int(np.prod([cfg.vel.n[i] for i in range(3)]))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ws_ptr = None
        self._ws = None
        if torch_workspace:
            nbytes = workspace_bytes(cfg)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) & ~255
        h = C.c_void_p()
        rc = lib().dvm_create(C.byref(cfg), ws_ptr, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise DvmError(rc, "dvm_create failed")
        self._h = h
        self._pending = {}

    @classmethod
    def from_case(cls, case, precision=F64, scheme=None, subcycles=None, **kw):
        cfg, keep = config_from_case(case, precision, scheme, subcycles)
        return cls(cfg, keep, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().dvm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc:
            raise DvmError(rc, lib().dvm_last_error(self._h).decode())

    # --------------------------------------------------------------- state
    def set_moments(self, U):
        t = self._torch
        if isinstance(U, t.Tensor):
            assert U.dtype == t.float64 and U.is_contiguous()
            self._check(lib().dvm_set_state_moments(self._h, C.c_void_p(U.data_ptr()),
                                                    1 if U.is_cuda else 0))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64).reshape(self.nm, self.nc)
            self._check(lib().dvm_set_state_moments(self._h, a.ctypes.data_as(C.c_void_p), 0))

    def set_primitive(self, rho, u, T):
        a = [np.ascontiguousarray(x, dtype=np.float64) for x in (rho, u, T)]
        ptrs = [x.ctypes.data_as(C.c_void_p) for x in a]
        self._check(lib().dvm_set_state_primitive(self._h, *ptrs, 0))

    def step(self, n=1):
        self._check(lib().dvm_step(self._h, int(n)))

    def step_async(self, n=1):
        self._check(lib().dvm_step_async(self._h, int(n)))

    def sync_status(self):
        self._check(lib().dvm_sync_status(self._h))

    # ----------------------------------------------------------- read-back
    def moments(self, out=None):
        t = self._torch
        if out is not None and isinstance(out, t.Tensor):
            assert out.dtype == t.float64 and out.is_contiguous()
            self._check(lib().dvm_moments(self._h, C.c_void_p(out.data_ptr()),
                                          1 if out.is_cuda else 0))
            return out
        a = np.zeros((self.nm, self.nc))
        self._check(lib().dvm_moments(self._h, a.ctypes.data_as(C.c_void_p), 0))
        return a

    def moments_async(self, out):
        """Enqueue a read-back of the moments after the steps enqueued so far into
        `out` (a float64 (d+2, N_c) torch tensor, pinned host or CUDA, or a numpy
        array); returns a ticket for moments_wait.  `out` is kept alive until then."""
        t = self._torch
        if isinstance(out, t.Tensor):
            assert out.dtype == t.float64 and out.is_contiguous() and out.numel() == self.nm * self.nc
            ptr, dev = out.data_ptr(), 1 if out.is_cuda else 0
        else:
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.nm * self.nc
            ptr, dev = out.ctypes.data, 0
        ticket = C.c_longlong()
        self._check(lib().dvm_moments_async(self._h, C.c_void_p(ptr), dev, C.byref(ticket)))
        self._pending[ticket.value] = out
        return ticket.value

    def moments_wait(self, ticket):
        """Block until read-back `ticket` is in its buffer; raises DvmError with the
        device status as that read-back's snapshot found it."""
        try:
            self._check(lib().dvm_moments_wait(self._h, int(ticket)))
        finally:
            for k in [k for k in self._pending if k <= ticket]:
                del self._pending[k]

    def f(self):
        a = np.zeros((self.nvel, self.nc))
        self._check(lib().dvm_get_f(self._h, a.ctypes.data_as(C.c_void_p), 0))
        return a

    def parts(self):
        shape = (self.nm, self.nc)
        UE, UM, Us = np.zeros(shape), np.zeros(shape), np.zeros(shape)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        self._check(lib().dvm_last_parts(self._h, p(UE), p(UM), p(Us)))
        return UE, UM, Us

    def info(self):
        dt, n, m = C.c_double(), C.c_longlong(), C.c_int()
        alpha = np.zeros(3)
        self._check(lib().dvm_info(self._h, C.byref(dt), C.byref(n), C.byref(m),
                                   alpha.ctypes.data_as(C.POINTER(C.c_double))))
        return {"dt": dt.value, "n": n.value, "m": m.value, "alpha": alpha}

    def offsets(self, n):
        width = max(self.cfg.vel.n[i] for i in range(self.d))
        out = np.zeros((self.d, width), dtype=np.int64)
        self._check(lib().dvm_offsets(self._h, int(n), out.ctypes.data_as(C.POINTER(C.c_longlong))))
        return out

    def save(self) -> bytes:
        n = C.c_size_t()
        self._check(lib().dvm_save(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lib().dvm_save(self._h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(lib().dvm_load(self._h, buf, len(blob)))

    def profile_begin(self):
        self._check(lib().dvm_profile_begin(self._h))

    def profile_end(self):
        """(summed kinetic-pass milliseconds, launches timed) since profile_begin."""
        ms, n = C.c_double(), C.c_int()
        self._check(lib().dvm_profile_end(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launches_per_step(self) -> int:
        n = C.c_int()
        self._check(lib().dvm_launches_per_step(self._h, C.byref(n)))
        return n.value

    def kinetic_kernel(self) -> str:
        """'generic' or 'window': the kinetic-pass kernel of this handle."""
        k = C.c_int()
        self._check(lib().dvm_kinetic_kernel(self._h, C.byref(k)))
        return ("generic", "window")[k.value]

    def kinetic_splits(self) -> int:
        """Velocity chunks of the kinetic pass (CTAs per target tile)."""
        k = C.c_int()
        self._check(lib().dvm_kinetic_splits(self._h, C.byref(k)))
        return k.value

    # --------------------------------------------------- learned regime path
    def learn_enable(self, mode=LEARN_GIVEN, mlp_precision=F32, thr=-3.0, check_every=0,
                     check_samples=256, veto_radius=2, seed=1212, shift=None, scale=None):
        c = _LearnConfig()
        c.mode, c.mlp_precision, c.thr = int(mode), int(mlp_precision), float(thr)
        c.check_every, c.check_samples, c.veto_radius = int(check_every), int(check_samples), int(veto_radius)
        c.seed = int(seed)
        c.feat_shift[:] = [float(x) for x in (np.zeros(NFEAT) if shift is None else shift)]
        c.feat_scale[:] = [float(x) for x in (np.ones(NFEAT) if scale is None else scale)]
        self._check(lib().dvm_learn_enable(self._h, C.byref(c)))

    def learn_disable(self):
        c = _LearnConfig()
        c.mode = LEARN_OFF
        self._check(lib().dvm_learn_enable(self._h, C.byref(c)))

    def learn_set_params(self, P):
        a = np.ascontiguousarray(P, dtype=np.float32)
        assert a.size == MLP_NPARAM
        self._check(lib().dvm_learn_set_params(self._h, a.ctypes.data_as(C.c_void_p)))

    def learn_set_flags(self, flags):
        a = np.ascontiguousarray(np.asarray(flags) != 0, dtype=np.uint8)
        assert a.size == self.nc
        self._check(lib().dvm_learn_set_flags(self._h, a.ctypes.data_as(C.c_void_p)))

    def learn_flags(self):
        a = np.zeros(self.nc, dtype=np.uint8)
        self._check(lib().dvm_learn_flags(self._h, a.ctypes.data_as(C.c_void_p)))
        return a

    def learn_predictions(self):
        a = np.zeros(self.nc, dtype=np.float32)
        self._check(lib().dvm_learn_predictions(self._h, a.ctypes.data_as(C.c_void_p)))
        return a

    def learn_stats(self) -> dict:
        st = _LearnStats()
        self._check(lib().dvm_learn_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _LearnStats._fields_}

    def learn_step_checked(self, cells):
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros(cells.size, dtype=np.float32)
        self._check(lib().dvm_learn_step_checked(self._h, int(cells.size),
                                                 cells.ctypes.data_as(C.c_void_p),
                                                 out.ctypes.data_as(C.c_void_p)))
        return out

    def features(self):
        """The ten regime features of the current state, shape (Nc, 10)."""
        a = np.zeros((self.nc, NFEAT), dtype=np.float32)
        self._check(lib().dvm_features(self._h, a.ctypes.data_as(C.c_void_p)))
        return a

    def noneq(self):
        """log10 of ||f - E[U]||_1 / ||E[U]||_1 per cell (true f)."""
        a = np.zeros(self.nc, dtype=np.float32)
        self._check(lib().dvm_noneq(self._h, a.ctypes.data_as(C.c_void_p)))
        return a


class Mlp:
    """The regime network on device data (dvm_mlp_*): X is a CUDA FP32 tensor of
    shape (n, 10), targets and outputs CUDA FP32 tensors of shape (n,)."""

    def __init__(self, precision=F32, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libdvm needs a CUDA GPU; no CPU fallback exists")
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = lib().dvm_mlp_create(int(precision), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise DvmError(rc, "dvm_mlp_create failed")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().dvm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc:
            raise DvmError(rc, "dvm_mlp call failed")

    def set_params(self, P):
        a = np.ascontiguousarray(P, dtype=np.float32)
        assert a.size == MLP_NPARAM
        self._check(lib().dvm_mlp_set_params(self._h, a.ctypes.data_as(C.c_void_p)))

    def params(self):
        a = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(lib().dvm_mlp_get_params(self._h, a.ctypes.data_as(C.c_void_p)))
        return a

    def _dev(self, X, dtype):
        t = self._torch
        X = t.as_tensor(X, dtype=dtype, device="cuda").contiguous()
        return X

    def forward(self, X):
        t = self._torch
        X = self._dev(X, t.float32)
        y = t.empty(X.shape[0], dtype=t.float32, device="cuda")
        self._check(lib().dvm_mlp_forward(self._h, X.shape[0], C.c_void_p(X.data_ptr()),
                                          C.c_void_p(y.data_ptr())))
        return y

    def loss_grad(self, X, y):
        t = self._torch
        X, y = self._dev(X, t.float32), self._dev(y, t.float32)
        g = t.empty(MLP_NPARAM, dtype=t.float64, device="cuda")
        loss = C.c_double()
        self._check(lib().dvm_mlp_loss_grad(self._h, X.shape[0], C.c_void_p(X.data_ptr()),
                                            C.c_void_p(y.data_ptr()), C.c_void_p(g.data_ptr()),
                                            C.byref(loss)))
        return loss.value, g.cpu().numpy()

    def train(self, X, y, epochs=10, batch=4096, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
              seed=1212):
        t = self._torch
        X, y = self._dev(X, t.float32), self._dev(y, t.float32)
        c = _TrainConfig()
        c.epochs, c.batch, c.lr, c.beta1, c.beta2, c.eps, c.seed = \
            int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps), int(seed)
        loss = C.c_double()
        self._check(lib().dvm_mlp_train(self._h, X.shape[0], C.c_void_p(X.data_ptr()),
                                        C.c_void_p(y.data_ptr()), C.byref(c), C.byref(loss)))
        return loss.value


class Batch:
    """Many independent 1D-1V and 2D-2V cases advanced together (dvm_batch_*).
    Moments are packed: `rows` rows (3 if every case is 1D, else 4) over all
    cells, case after case; a case of dimension d fills its first d + 2 rows."""

    def __init__(self, cases, precision=F32, scheme=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libdvm needs a CUDA GPU; no CPU fallback exists")
        self._torch = torch
        arr = (_Config * len(cases))()
        self._keep = []
        for i, case in enumerate(cases):
            cfg, keep = config_from_case(case, precision, scheme)
            arr[i] = cfg
            self._keep += keep
        self._cfgs = arr
        self.ncases = len(cases)
        self.dims = [int(c.d) for c in cases]
        self.nx = [int(np.prod(c.nx)) for c in cases]     # cells of each case
        self.nv = [int(np.prod(c.nv)) for c in cases]     # velocities of each case
        self.offsets = np.concatenate([[0], np.cumsum(self.nx)]).astype(int)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        rc = lib().dvm_batch_create(arr, len(cases), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc:
            raise DvmError(rc, "dvm_batch_create failed")
        self._h = h
        self._pending = {}
        cells, pts, rows = C.c_longlong(), C.c_longlong(), C.c_int()
        lib().dvm_batch_sizes(h, C.byref(cells), C.byref(pts))
        lib().dvm_batch_moment_rows(h, C.byref(rows))
        self.ncells, self.npoints, self.rows = cells.value, pts.value, rows.value

    def close(self):
        if getattr(self, "_h", None):
            lib().dvm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _check(self, rc):
        if rc:
            raise DvmError(rc, lib().dvm_batch_last_error(self._h).decode())

    def pack(self, per_case):
        """Pack a list of (d_i + 2, N_cells,i) moment arrays into the batch layout."""
        out = np.zeros((self.rows, self.ncells))
        for i, U in enumerate(per_case):
            out[:U.shape[0], self.offsets[i]:self.offsets[i + 1]] = U
        return out

    def set_moments(self, U):
        t = self._torch
        if isinstance(U, t.Tensor):
            self._check(lib().dvm_batch_set_state_moments(self._h, C.c_void_p(U.data_ptr()),
                                                          1 if U.is_cuda else 0))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64)
            self._check(lib().dvm_batch_set_state_moments(self._h, a.ctypes.data_as(C.c_void_p), 0))

    def step(self, n=1):
        self._check(lib().dvm_batch_step(self._h, int(n)))

    def step_async(self, n=1):
        self._check(lib().dvm_batch_step_async(self._h, int(n)))

    def sync_status(self):
        self._check(lib().dvm_batch_sync_status(self._h))

    def moments(self, out=None):
        t = self._torch
        if out is not None and isinstance(out, t.Tensor):
            self._check(lib().dvm_batch_moments(self._h, C.c_void_p(out.data_ptr()),
                                                1 if out.is_cuda else 0))
            return out
        a = np.zeros((self.rows, self.ncells))
        self._check(lib().dvm_batch_moments(self._h, a.ctypes.data_as(C.c_void_p), 0))
        return a

    def moments_async(self, out):
        """Pipelined read-back of the packed moments into `out` (float64 (rows, cells):
        pinned host or CUDA torch tensor, or numpy array); returns a ticket."""
        t = self._torch
        if isinstance(out, t.Tensor):
            assert out.dtype == t.float64 and out.is_contiguous() and out.numel() == self.rows * self.ncells
            ptr, dev = out.data_ptr(), 1 if out.is_cuda else 0
        else:
            assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.rows * self.ncells
            ptr, dev = out.ctypes.data, 0
        ticket = C.c_longlong()
        self._check(lib().dvm_batch_moments_async(self._h, C.c_void_p(ptr), dev, C.byref(ticket)))
        self._pending[ticket.value] = out
        return ticket.value

    def moments_wait(self, ticket):
        try:
            self._check(lib().dvm_batch_moments_wait(self._h, int(ticket)))
        finally:
            for k in [k for k in self._pending if k <= ticket]:
                del self._pending[k]

    def case_moments(self, U, i):
        return U[:self.dims[i] + 2, self.offsets[i]:self.offsets[i + 1]]

    def f(self, i):
        a = np.zeros((self.nv[i], self.nx[i]))
        self._check(lib().dvm_batch_get_f(self._h, int(i), a.ctypes.data_as(C.c_void_p)))
        return a

    def info(self):
        n = C.c_longlong()
        m = np.zeros(self.ncases, dtype=np.int32)
        a = np.zeros(self.ncases)
        self._check(lib().dvm_batch_info(self._h, C.byref(n), m.ctypes.data_as(C.c_void_p),
                                         a.ctypes.data_as(C.c_void_p)))
        return {"n": n.value, "m": m, "alpha": a}

    def set_tiling(self, threads, cells_per_thread, vchunks=1, ctas_per_sm=0):
        self._check(lib().dvm_batch_set_tiling(self._h, int(threads), int(cells_per_thread), int(vchunks),
                                               int(ctas_per_sm)))

    def autotune(self):
        """(threads, cells per thread, velocity chunks, CTAs per SM, ms) of the
        fastest kinetic-pass launch, which the batch keeps."""
        t, c, v, o, ms = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
        self._check(lib().dvm_batch_autotune(self._h, C.byref(t), C.byref(c), C.byref(v), C.byref(o),
                                             C.byref(ms)))
        return t.value, c.value, v.value, o.value, ms.value

    def kinetic_ms(self, nsteps=3):
        ms = C.c_double()
        self._check(lib().dvm_batch_kinetic_ms(self._h, int(nsteps), C.byref(ms)))
        return ms.value


def autotune_cached(batch: "Batch", cases, precision, scheme) -> dict:
    """Tile of the batched kinetic pass from a JSON cache keyed by the batch's
    shapes; runs dvm_batch_autotune on a miss and records the result.  The cache
    lives in $DVM_CACHE_DIR or ~/.cache/dvm (skipped if not writable)."""
    import hashlib
    import json
    sig = hashlib.sha256(json.dumps([[int(c.d), list(map(int, c.nx)), list(map(int, c.nv))] for c in cases] +
                                    [precision, scheme, 2]).encode()).hexdigest()[:20]
    d = os.environ.get("DVM_CACHE_DIR", os.path.join(os.path.expanduser("~"), ".cache", "dvm"))
    path = os.path.join(d, "batch_autotune.json")
    table = {}
    try:
        with open(path) as fh:
            table = json.load(fh)
    except (OSError, ValueError):
        table = {}
    if sig in table:
        e = table[sig]
        batch.set_tiling(e["threads"], e["cells_per_thread"], e["vchunks"], e["ctas_per_sm"])
        return dict(e, cached=True)
    t, c, v, o, ms = batch.autotune()
    table[sig] = {"threads": t, "cells_per_thread": c, "vchunks": v, "ctas_per_sm": o, "kinetic_ms": ms}
    try:
        os.makedirs(d, exist_ok=True)
        with open(path, "w") as fh:
            json.dump(table, fh, indent=1)
    except OSError:
        pass
    return dict(table[sig], cached=False)
