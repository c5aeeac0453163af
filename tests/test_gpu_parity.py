"""GPU-vs-oracle parity through the C ABI (libdvm.so via the ctypes binding).

Tolerances: shift indexing bit-exact; moments 1e-12 relative
in the FP64 build and 1e-5 relative in the FP32 build; BF16 storage reports its
error against a stated bound.  A moment row's error is measured against
max(|U_i|_inf, |rho|_inf): the scale of a sum of f_k m_k with |m_k| = O(1), which
keeps near-zero momentum rows meaningful.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1212_0204_gb300 import workloads as W
from tests.helpers import conserved, grid, velocity_indices

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1212_0204_gb300 import dvm  # noqa: E402


def moment_err(Ug, Uo):
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    return (np.abs(Ug - Uo).max(axis=1) / scale).max()


def gpu_run(case, steps, precision=dvm.F64, scheme=None, subcycles=None, U0=None):
    s = dvm.Solver.from_case(case, precision=precision, scheme=scheme, subcycles=subcycles)
    s.set_moments(conserved(case) if U0 is None else U0)
    s.step(steps)
    return s


def small_cases():
    """Reduced-size versions of the workloads: several tiles and ragged tails."""
    sod = W.sod_1d(nx=203, nv=32, tau=1e-4)
    sod2 = W.sod_1d(nx=150, nv=32, tau=1e-2, p=3)
    quad = W.quadrant_2d(n=37, nv=16, tau=1e-3, steps=4, dv=0.7)
    wave = W.density_wave_3d(n=9, nv=8, tau=1e-4, steps=3, dv=1.2)
    shear = W.shear_layer_2d(n=33, nv=10, steps=3, dv=1.0)
    return {"sod_1d": (sod, 6), "sod_1d_p3": (sod2, 7), "quadrant_2d": (quad, 4),
            "density_wave_3d": (wave, 3), "shear_layer_2d_taufield": (shear, 3)}


CASES = small_cases()


@pytest.mark.parametrize("p", [1, 3, 13])
def test_offsets_are_bit_exact(p):
    case = W.sod_1d(nx=50, nv=32, p=p)
    s = dvm.Solver.from_case(case)
    kk = np.arange(-16, 16)
    for n in (0, 1, 2, 7, 100, 12345):
        got = s.offsets(n)[0]
        want = np.array([oracle.offset(int(k), n, p) for k in kk])
        assert np.array_equal(got, want), (p, n)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("scheme", [dvm.HOFKS, dvm.FKS])
def test_fp64_matches_oracle(name, scheme):
    case, steps = CASES[name]
    orc = oracle.Scheme(grid(case, scheme), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(steps)
    g = gpu_run(case, steps, dvm.F64, scheme)
    assert moment_err(g.moments(), orc.moments()) <= 1e-12
    fo = orc.f()
    assert np.abs(g.f() - fo).max() <= 1e-12 * np.abs(fo).max()


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_matches_oracle(name):
    case, steps = CASES[name]
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(steps)
    g = gpu_run(case, steps, dvm.F32)
    assert moment_err(g.moments(), orc.moments()) <= 1e-5


@pytest.mark.parametrize("name", ["quadrant_2d", "density_wave_3d"])
def test_bf16_storage_error_is_bounded(name):
    """BF16 storage (8-bit mantissa, relative rounding 2^-9 per store): the moment
    error against the FP64 oracle stays within a few rounding units."""
    case, steps = CASES[name]
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(steps)
    g = gpu_run(case, steps, dvm.BF16S)
    err = moment_err(g.moments(), orc.moments())
    assert err <= 8 * 2.0 ** -9, err


def test_hofks_parts_match_oracle():
    case, steps = CASES["quadrant_2d"]
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(steps)
    g = gpu_run(case, steps, dvm.F64)
    for a, b in zip(g.parts(), orc.parts()):
        assert moment_err(a, b) <= 1e-12
    gi, oi = g.info(), orc.info()
    # the integer decision (Euler sub-steps) must agree; alpha itself is computed
    # from moments that differ at round-off between the two sides
    assert gi["m"] == oi["m"] and gi["n"] == oi["n"]
    np.testing.assert_allclose(gi["alpha"][:2], oi["alpha"][:2], rtol=1e-13, atol=0)


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("precision", [dvm.F64, dvm.F32, dvm.BF16S])
def test_free_transport_is_bit_exact(p, precision):
    """tau = inf: the GPU's f after n steps is its own f^0 shifted by the exact
    offsets, bit for bit, in every storage precision."""
    case = W.quadrant_2d(n=19, nv=8, tau=np.inf, steps=5, dv=0.9)
    case.p = p
    s = dvm.Solver.from_case(case, precision=precision)
    s.set_moments(conserved(case))
    f0 = s.f().reshape(case.nvel, 19, 19)
    n = 6
    s.step(n)
    g = grid(case)
    kk = velocity_indices(g)
    expect = np.empty_like(f0)
    for k in range(case.nvel):
        ox, oy = oracle.offset(int(kk[0, k]), n, p), oracle.offset(int(kk[1, k]), n, p)
        expect[k] = np.roll(np.roll(f0[k], oy, axis=0), ox, axis=1)
    assert np.array_equal(s.f().reshape(expect.shape), expect)


def test_free_transport_outflow_is_bit_exact():
    case = W.sod_1d(nx=41, nv=16, tau=np.inf, steps=5)
    s = dvm.Solver.from_case(case, precision=dvm.F64)
    s.set_moments(conserved(case))
    f0 = s.f()
    n = 5
    s.step(n)
    c = np.arange(41)
    expect = np.stack([f0[k, np.clip(c - oracle.offset(-8 + k, n, 1), 0, 40)] for k in range(16)])
    assert np.array_equal(s.f(), expect)


@pytest.mark.parametrize("precision,tol", [(dvm.F64, 1e-13), (dvm.F32, 1e-6)])
def test_periodic_conservation_on_gpu(precision, tol):
    case = W.quadrant_2d(n=40, nv=16, tau=1e-3, steps=5, dv=0.8)
    s = dvm.Solver.from_case(case, precision=precision)
    U0 = conserved(case)
    s.set_moments(U0)
    s.step(5)
    U = s.moments()
    scale = np.abs(U0).sum(1)
    scale[1:3] = scale[0]
    assert np.all(np.abs(U.sum(1) - U0.sum(1)) <= tol * scale)


def test_uniform_equilibrium_is_a_fixed_point_on_gpu():
    case = W.quadrant_2d(n=16, nv=16, tau=1e-3, steps=3, dv=0.8)
    U0 = np.tile(np.array([[1.0], [0.1], [-0.2], [1.3]]), (1, case.ncells))
    s = dvm.Solver.from_case(case)
    s.set_moments(U0)
    f0 = s.f()
    s.step(3)
    assert np.abs(s.f() - f0).max() <= 1e-14 * np.abs(f0).max()
    assert np.abs(s.moments() - U0).max() <= 1e-14 * np.abs(U0).max()


@pytest.mark.parametrize("precision", [dvm.F64, dvm.F32])
def test_checkpoint_resume_is_bit_exact(precision):
    case = W.sod_1d(nx=64, nv=32, tau=1e-3)
    a = dvm.Solver.from_case(case, precision=precision)
    a.set_moments(conserved(case))
    a.step(3)
    blob = a.save()
    a.step(4)
    b = dvm.Solver.from_case(case, precision=precision)
    b.load(blob)
    b.step(4)
    assert np.array_equal(a.moments(), b.moments())
    assert np.array_equal(a.f(), b.f())
    assert a.info()["n"] == b.info()["n"] == 7


def test_nonphysical_state_is_reported():
    case = W.sod_1d(nx=20, nv=16)
    s = dvm.Solver.from_case(case)
    U = conserved(case)
    U[0, 3] = -1.0
    with pytest.raises(dvm.DvmError) as e:
        s.set_moments(U)
    assert e.value.code == dvm.ERR_NONPHYSICAL


def test_primitive_and_moment_initialisation_agree():
    case = CASES["density_wave_3d"][0]
    a = dvm.Solver.from_case(case)
    a.set_primitive(case.rho, case.u, case.T)
    b = dvm.Solver.from_case(case)
    b.set_moments(conserved(case))
    assert moment_err(a.moments(), b.moments()) <= 1e-15
    assert np.abs(a.f() - b.f()).max() <= 1e-14 * np.abs(b.f()).max()


@pytest.mark.parametrize("case", [
    W.sod_1d(nx=64, nv=32, tau=0.0),
    W.quadrant_2d(n=20, nv=16, tau=0.0, steps=3, dv=0.7),
], ids=["sod_tau0", "quadrant_tau0"])
def test_tau_zero_matches_oracle(case):
    """lambda = 0 exactly (the fluid limit: HOFKS reduces to the Euler scheme)."""
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(3)
    g = gpu_run(case, 3, dvm.F64)
    assert moment_err(g.moments(), orc.moments()) <= 1e-12


@pytest.mark.parametrize("case,precision,tol", [
    (W.sod_1d(nx=3, nv=8, tau=1e-3, dv=1.0), dvm.F64, 1e-12),          # three cells
    (W.quadrant_2d(n=5, nv=8, tau=1e-3, steps=2, dv=1.0), dvm.F64, 1e-12),  # 5 x 5, one tile
    (W.sod_1d(nx=40, nv=256, tau=1e-3, dv=0.05), dvm.F64, 1e-12),     # 256 velocities (maximum)
    (W.quadrant_2d(n=33, nv=16, tau=1e-3, steps=2, dv=0.7), dvm.F32, 1e-5),  # ragged x and y tails
], ids=["three_cells", "five_by_five", "max_velocities", "ragged_window"])
def test_edge_sizes_match_oracle(case, precision, tol):
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(2)
    g = gpu_run(case, 2, precision)
    assert moment_err(g.moments(), orc.moments()) <= tol


@pytest.mark.parametrize("make", [
    lambda: W.quadrant_2d(n=128, nv=32, tau=1e-3, steps=4),
    lambda: W.density_wave_3d(n=32, nv=24, tau=1e-4, steps=2, dv=0.5),
])
def test_shape_compiled_pass_equals_runtime_pass(make, monkeypatch):
    """The kinetic pass compiled for a configured shape (extents as constants)
    gives bit-identical moments and f (2D) to the same kernel with run-time
    extents.  In 3D the configured shapes run the CTA-shared-slot kernel, which
    forms the same values but adds the moment sums in another order (FP32 over
    the split's pairs): moments within 1e-6 of the moment scale."""
    case = make()
    out = []
    for mode in ("1", "0"):
        monkeypatch.setenv("DVM_FIXED_SHAPES", mode)
        s = dvm.Solver.from_case(case, precision=dvm.F32)
        s.set_moments(conserved(case))
        s.step(case.steps)
        out.append((s.moments(), s.f() if case.d == 2 else None))
        s.close()
    if case.d == 2:
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
    else:
        assert moment_err(out[0][0], out[1][0]) <= 1e-6


@pytest.mark.parametrize("tau", [1e-4, 0.1], ids=["fluid", "kinetic"])
@pytest.mark.parametrize("scheme", [dvm.HOFKS, dvm.FKS])
def test_3d_bench_velocity_grid_with_velocity_splits_matches_oracle(scheme, tau):
    """3D-3V at the benchmark's velocity grid (24^3 velocities, dv = 0.5) on 16^3
    cells: the windowed pass splits the kz planes of every target tile over several
    CTAs, whose FP64 partial moment sums the end-of-step kernel adds.  FP32 f against
    the FP64 oracle over 2 steps: moments at 1e-5, f element by element at 1e-5 of
    max |f|.  tau = 1e-4 is the benchmark's (lambda = 0 at this cell size: the
    relaxed part only); tau = 0.1 gives lambda = 0.29, so the transported
    lambda f part is exercised as well."""
    case = W.density_wave_3d(n=16, nv=24, tau=tau, steps=2, dv=0.5)
    orc = oracle.Scheme(grid(case, scheme), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(2)
    g = gpu_run(case, 2, dvm.F32, scheme)
    assert g.kinetic_kernel() == "window"
    assert g.kinetic_splits() > 1
    assert moment_err(g.moments(), orc.moments()) <= 1e-5
    fo = orc.f()
    assert np.abs(g.f() - fo).max() <= 1e-5 * np.abs(fo).max()
    if scheme == dvm.HOFKS:
        # U_E, U_M, U_* on the scale of the moments (U_* = 0 when lambda = 0)
        Uo = orc.moments()
        scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
        for a, b in zip(g.parts(), orc.parts()):
            assert (np.abs(a - b).max(axis=1) / scale).max() <= 1e-5


@pytest.mark.parametrize("tau", [1e-4, 0.1], ids=["fluid", "kinetic"])
def test_3d_bf16_storage_at_the_bench_velocity_grid_is_bounded(tau):
    """BF16 storage on the 3D pass at the benchmark's velocity grid (16^3 x 24^3,
    several velocity splits, the single-quadratic form): after 2 steps the moments
    stay within a few BF16 rounding units (2^-9 relative per store) of the FP64
    oracle, and f within 4 x 2^-9 of max |f| (a stored value is rounded once per
    step)."""
    case = W.density_wave_3d(n=16, nv=24, tau=tau, steps=2, dv=0.5)
    orc = oracle.Scheme(grid(case, dvm.HOFKS), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(2)
    g = gpu_run(case, 2, dvm.BF16S)
    assert g.kinetic_kernel() == "window"
    assert g.kinetic_splits() > 1
    assert moment_err(g.moments(), orc.moments()) <= 8 * 2.0 ** -9
    fo = orc.f()
    assert np.abs(g.f() - fo).max() <= 4 * 2.0 ** -9 * np.abs(fo).max()


@pytest.mark.parametrize("tau", [0.05, None], ids=["kinetic", "taufield"])
def test_3d_shared_slot_kernel_matches_oracle(tau, monkeypatch):
    """The 3D kinetic pass of the configured shapes (the CTA folds each pair's
    source rows once into shared memory, four warps stacked in y share them, moment
    sums in registers) at 32^3 x 8^3 against the FP64 oracle over 3 steps: moments,
    U_E, U_M, U_* at 1e-5 of the moment scale, f element by element at 1e-5 of
    max |f|; lambda = 0.54, then a tau field with lambda from 0 to 0.91."""
    monkeypatch.setenv("DVM_FIXED_SHAPES", "1")
    case = W.density_wave_3d(n=32, nv=8, tau=0.05 if tau else 1e-2, steps=3, dv=1.0)
    if tau is None:
        xc = (np.arange(32) + 0.5) / 32
        Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
        r = 0.5 * (1 + np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(2 * np.pi * Z))
        case = dataclasses.replace(case, tau=(10.0 ** (-4 + 4 * r)).ravel() * 0.375)
    orc = oracle.Scheme(grid(case, dvm.HOFKS), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(3)
    g = gpu_run(case, 3, dvm.F32)
    assert g.kinetic_kernel() == "window"
    Uo = orc.moments()
    assert moment_err(g.moments(), Uo) <= 1e-5
    fo = orc.f()
    assert np.abs(g.f() - fo).max() <= 1e-5 * np.abs(fo).max()
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    for a, b in zip(g.parts(), orc.parts()):
        assert (np.abs(a - b).max(axis=1) / scale).max() <= 1e-5


def _wave_3d_tau_field():
    """12^3 x 8^3 density wave with tau = 10^(-4 + 4 r), r = (1 + sin 2pi x cos 2pi y
    cos 2pi z) / 2: lambda = exp(-dt/tau) from 0 to 0.88 across the box."""
    case = W.density_wave_3d(n=12, nv=8, tau=1e-2, steps=3, dv=1.0)
    xc = (np.arange(12) + 0.5) / 12
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    r = 0.5 * (1 + np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) * np.cos(2 * np.pi * Z))
    return dataclasses.replace(case, tau=(10.0 ** (-4 + 4 * r)).ravel())


def _odd_box_3d():
    """37 x 6 x 5 periodic box (ragged x tile; N_y and N_z below the 8 velocities per
    axis, so sources wrap more than once) with an off-centre velocity grid (k from
    -3, -5, -4) and u = (0.3, -0.2, 0.1)."""
    nx, dx = (37, 6, 5), 1.0 / 37
    xs = [(np.arange(n) + 0.5) * dx for n in nx]
    Z, Y, X = (a.ravel() for a in np.meshgrid(xs[2], xs[1], xs[0], indexing="ij"))
    L = [n * dx for n in nx]
    rho = 1 + 0.2 * np.sin(2 * np.pi * X / L[0]) * np.cos(2 * np.pi * Y / L[1]) * np.cos(2 * np.pi * Z / L[2])
    u = np.stack([np.full_like(X, 0.3), np.full_like(X, -0.2), np.full_like(X, 0.1)])
    T = 1 + 0.1 * np.sin(2 * np.pi * X / L[0])
    return W.Case("odd_box_3d", 3, nx, dx, (8, 8, 8), (-3, -5, -4), 1.0, 1, (W.PERIODIC,) * 3, 0.05,
                  rho, u, T, 3, W.HOFKS)


@pytest.mark.parametrize("make", [
    lambda: W.density_wave_3d(n=12, nv=8, tau=0.05, steps=3, dv=1.0),
    _wave_3d_tau_field,
    _odd_box_3d,
], ids=["wave_3d_kinetic", "wave_3d_taufield", "odd_box_offset_velocities"])
def test_windowed_3d_linear_term_moments_match_oracle(make):
    """3D HOFKS on the windowed pass keeps one quadratic per source for the deferred
    and the moment-matching terms together, sums the new value and the Maxwellian
    part only, and adds the moments of the transported mu''.m term from separate
    per-axis passes over the cells; U_M and U_* follow from these.  Against the FP64
    oracle over 3 steps: moments, U_E, U_M and U_* at 1e-5 of the moment scale, f
    element by element at 1e-5 of max |f|; lambda = 0.19 everywhere, then a tau
    field with lambda from 0 to 0.88, then an odd-shaped box with an off-centre
    velocity grid."""
    case = make()
    orc = oracle.Scheme(grid(case, dvm.HOFKS), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(3)
    g = gpu_run(case, 3, dvm.F32)
    assert g.kinetic_kernel() == "window"
    Uo = orc.moments()
    assert moment_err(g.moments(), Uo) <= 1e-5
    fo = orc.f()
    assert np.abs(g.f() - fo).max() <= 1e-5 * np.abs(fo).max()
    scale = np.maximum(np.abs(Uo).max(axis=1), np.abs(Uo[0]).max())
    for a, b in zip(g.parts(), orc.parts()):
        assert (np.abs(a - b).max(axis=1) / scale).max() <= 1e-5


@pytest.mark.parametrize("n", [64, 96])
def test_3d_shape_compiled_pass_equals_runtime_pass_at_bench_sizes(n, monkeypatch):
    """The 3D kinetic pass compiled for the 64^3 and 96^3 x 24^3 shapes (the
    CTA-shared-slot kernel behind the 3D benchmark lines) agrees with the per-thread
    window kernel with run-time extents over 2 steps: moments, U_E, U_M and U_*
    within 1e-6 of the moment scale (the same values, moment sums added in another
    order); f itself is compared through the moments (at 96^3 it is 49 GB)."""
    case = W.density_wave_3d(n=n, nv=24, tau=1e-4, steps=2, dv=0.5)
    out = []
    for mode in ("1", "0"):
        monkeypatch.setenv("DVM_FIXED_SHAPES", mode)
        s = dvm.Solver.from_case(case, precision=dvm.F32)
        s.set_moments(conserved(case))
        s.step(2)
        out.append((s.moments(), s.parts()))
        s.close()
        del s
    U = out[1][0]
    scale = np.maximum(np.abs(U).max(axis=1), np.abs(U[0]).max())
    assert moment_err(out[0][0], U) <= 1e-6
    for a, b in zip(out[0][1], out[1][1]):
        assert (np.abs(a - b).max(axis=1) / scale).max() <= 1e-6


@pytest.mark.parametrize("n", [9, 21])
def test_3d_z_marching_euler_agrees_with_the_per_face_kernel(n, monkeypatch):
    """The 3D Euler sub-steps marching along z (split fluxes per staged cell, five-
    plane ring) and the per-face kernel (each face from its four staged states) are
    two roundings of the same Eq. discmom update: FP64 U_E and moments to 1e-13 of
    their scale, the same sub-step count (21^3: ragged x and y tiles, several z
    chunks)."""
    case = W.density_wave_3d(n=n, nv=8, tau=1e-4, steps=3, dv=1.2)
    out = []
    for kernel in ("0", "1"):
        monkeypatch.setenv("DVM_EULER_KERNEL", kernel)
        s = gpu_run(case, 3, dvm.F64)
        out.append((s.moments(), s.parts()[0], s.info()["m"]))
        s.close()
    scale = np.abs(out[1][0]).max(axis=1, keepdims=True)
    assert (np.abs(out[0][0] - out[1][0]) / scale).max() <= 1e-13
    assert (np.abs(out[0][1] - out[1][1]) / scale).max() <= 1e-13
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("make", [
    lambda: W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=2),
    lambda: W.density_wave_3d(n=64, nv=24, tau=1e-2, steps=2, dv=0.5),
], ids=["quadrant_256", "wave_3d_64"])
def test_bf16_shape_compiled_pass_equals_runtime_pass(make, monkeypatch):
    """BF16 storage at the configured shapes (2D 256^2 x 32^2, 3D 64^3 x 24^3): the
    kernel compiled with the extents as constants gives moments (and f, in 2D)
    bit-identical to the kernel with run-time extents over 2 steps."""
    case = make()
    out = []
    for mode in ("1", "0"):
        monkeypatch.setenv("DVM_FIXED_SHAPES", mode)
        s = dvm.Solver.from_case(case, precision=dvm.BF16S)
        s.set_moments(conserved(case))
        s.step(case.steps)
        out.append((s.moments(), s.f() if case.d == 2 else None))
        s.close()
        del s
    assert np.array_equal(out[0][0], out[1][0])
    if case.d == 2:
        assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("make", [
    lambda: W.quadrant_2d(n=36, nv=16, tau=1e-3, steps=3, dv=0.7),
    lambda: W.density_wave_3d(n=10, nv=8, tau=1e-2, steps=2, dv=1.2),
], ids=["quadrant_36", "wave_3d_10"])
def test_bf16_staged_loads_equal_direct_loads(make, monkeypatch):
    """BF16 storage with N_x even stages the 4-byte word holding each value and
    takes the half named by the parity of its x piece: the same values as the
    direct 2-byte loads (DVM_WIN_ASYNC=0), so moments and f agree bit for bit;
    and the error against the FP64 oracle stays within the BF16 bound."""
    case = make()
    out = []
    for mode in ("1", "0"):
        monkeypatch.setenv("DVM_WIN_ASYNC", mode)
        s = gpu_run(case, case.steps, dvm.BF16S)
        out.append((s.moments(), s.f()))
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    orc = oracle.Scheme(grid(case), tau=case.tau)
    orc.set_moments(conserved(case))
    orc.step(case.steps)
    assert moment_err(out[0][0], orc.moments()) <= 8 * 2.0 ** -9


def test_bf16_free_transport_with_staged_loads_is_bit_exact():
    case = W.quadrant_2d(n=20, nv=8, tau=np.inf, steps=5, dv=0.9)
    s = dvm.Solver.from_case(case, precision=dvm.BF16S)
    s.set_moments(conserved(case))
    f0 = s.f().reshape(case.nvel, 20, 20)
    s.step(5)
    kk = velocity_indices(grid(case))
    expect = np.empty_like(f0)
    for k in range(case.nvel):
        ox, oy = oracle.offset(int(kk[0, k]), 5, 1), oracle.offset(int(kk[1, k]), 5, 1)
        expect[k] = np.roll(np.roll(f0[k], oy, axis=0), ox, axis=1)
    assert np.array_equal(s.f().reshape(expect.shape), expect)


@pytest.mark.parametrize("make", [
    lambda: W.quadrant_2d(n=45, nv=12, tau=1e-3, steps=3, dv=0.9),
    lambda: W.sod_1d(nx=300, nv=32, tau=1e-4),
], ids=["quadrant_2d", "sod_1d"])
@pytest.mark.parametrize("precision", [dvm.F64, dvm.F32])
def test_euler_kernels_agree_bit_for_bit(make, precision, monkeypatch):
    """The two-phase Euler kernel (each cell computes its own faces) with 32 x 32
    tiles (the default for FP32 2D grids this small) and with 32 x 4 tiles, and
    the four-phase one (faces computed once, shared) evaluate the same
    expressions: bit-identical U_E and moments (45 x 45 cells: ragged tiles)."""
    case = make()
    out = []
    for kernel, tall in (("0", "1"), ("0", "0"), ("2", "1")):
        monkeypatch.setenv("DVM_EULER_KERNEL", kernel)
        monkeypatch.setenv("DVM_EULER_TALL", tall)
        s = gpu_run(case, 3, precision)
        out.append((s.moments(), s.parts()[0], s.info()["m"]))
        s.close()
    for o in out[1:]:
        assert np.array_equal(out[0][0], o[0]) and np.array_equal(out[0][1], o[1])
        assert out[0][2] == o[2]
