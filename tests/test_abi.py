"""CPU checks of the boundary: libdvm.so builds, loads without a GPU and exports
every function include/dvm.h declares; the binding's list agrees with the header;
the header is plain C99 that a C program compiles (-pedantic -Werror) and links
against libdvm.so.  No compute call is made here."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dvm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def libdvm():
    from paper_1212_0204_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(libdvm):
    names = declared("dvm.h")
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(libdvm, n)]
    assert not missing, missing


def test_binding_lists_the_header(libdvm):
    from paper_1212_0204_gb300 import dvm
    assert sorted(dvm.EXPORTS) == declared("dvm.h")


def test_invalid_configuration_is_rejected_without_a_gpu(libdvm):
    from paper_1212_0204_gb300 import dvm
    cfg, _ = dvm.make_config(4, (8,), 0.1, (8,), (-4,), 0.5)
    with pytest.raises(dvm.DvmError):
        dvm.workspace_bytes(cfg)
    cfg, _ = dvm.make_config(1, (8,), 0.1, (300,), (-150,), 0.5)
    with pytest.raises(dvm.DvmError):
        dvm.workspace_bytes(cfg)
    cfg, _ = dvm.make_config(2, (64, 64), 1 / 64, (32, 32), (-16, -16), 0.4, precision=dvm.F32)
    n = dvm.workspace_bytes(cfg)
    assert n >= 64 * 64 * 32 * 32 * 4


def test_product_path_has_no_cpu_fallback():
    """The binding refuses to run without a GPU instead of computing on the CPU."""
    import torch
    from paper_1212_0204_gb300 import dvm, workloads
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        dvm.Solver.from_case(workloads.sod_1d(nx=16, nv=8))


def test_header_is_c99_and_a_c_program_links_and_calls_the_library(libdvm, tmp_path):
    """tests/abi_check.c fills a dvm_config as a C program would and asks for the
    workspace size (a host-only call): valid FP32/FP64 configs give the FP64 f twice
    the f bytes of FP32 plus the same per-cell buffers; degenerate and invalid ones
    (empty grid, no velocities, dx = 0, dv < 0, shift_den = 0, tau < 0 or NaN,
    mismatched faces, unknown scheme or precision, more than 256 velocities per
    dimension, a non-unit unused dimension) give DVM_ERR_ARG; 256 is accepted."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1212_0204_gb300 import build
    libdir = os.path.dirname(build.build())
    exe = tmp_path / "abi_check"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_check.c"),
                    "-L", libdir, "-ldvm", "-Wl,-rpath," + libdir, "-lm", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = {ln.split()[0]: [int(v) for v in ln.split()[1:]] for ln in out if ln.strip()}
    (rc32, b32), (rc64, b64) = rows["f32"], rows["f64"]
    assert rc32 == 0 and rc64 == 0
    f_bytes = 64 * 64 * 32 * 32
    assert b32 >= 4 * f_bytes and b64 - b32 >= 4 * f_bytes
    assert rows["bad_dim"][0] == -1 and rows["null"][0] == -1
    assert rows["tau_inf"][0] == 0
    bad = {k: v[0] for k, v in rows.items() if k.startswith("bad_")}
    assert len(bad) == 13 and all(v == -1 for v in bad.values()), bad
    assert rows["max_velocities"][0] == 0


def test_launch_plan_without_a_gpu(libdvm):
    """dvm_plan reports the kinetic-pass kernel and its velocity splits host-side, for
    152 SMs when no device is visible.  The configured 3D FP32 shapes (the
    CTA-shared-slot kernel, 32 x 16 targets per CTA, 3 CTAs per SM) take the divisor
    c <= 12 of N_v1 with the smallest ceil(w) / w (1 + 20 c / N_v), w = CTA waves: the
    last wave nearly full at little partial-sum traffic; other windowed shapes keep
    c <= 4; the FP64 tier runs the generic pass."""
    import math

    from paper_1212_0204_gb300 import dvm, workloads as W

    def plan(case, prec):
        cfg, keep = dvm.config_from_case(case, precision=prec)
        return dvm.plan(cfg)

    def tile_choice(n, v):
        tiles, resident, nvel = (n // 32) * (n // 16) * n, 152 * 3, v ** 3
        best = None
        for c in range(1, 13):
            if v % c or (c > 1 and 512 * nvel // c < 65536):
                continue
            w = tiles * c / resident
            cost = math.ceil(w) / w * (1 + 20 * c / nvel)
            if best is None or cost < best[0]:
                best = (cost, c)
        return best[1]

    for n in (96, 64):
        kind, sp = plan(W.density_wave_3d(n=n, nv=24, tau=1e-4, steps=1), dvm.F32)
        assert kind == "window" and sp == tile_choice(n, 24) and 24 % sp == 0
    assert plan(W.density_wave_3d(n=96, nv=24, tau=1e-4, steps=1), dvm.F32)[1] == 6
    assert plan(W.density_wave_3d(n=64, nv=24, tau=1e-4, steps=1), dvm.F32)[1] == 8
    # BF16 storage and unconfigured shapes: the per-thread window kernel's rule (c <= 4)
    kind, sp = plan(W.density_wave_3d(n=16, nv=24, tau=1e-4, steps=1), dvm.BF16S)
    assert kind == "window" and 1 <= sp <= 4 and 24 % sp == 0
    assert plan(W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=1), dvm.F32) == ("window", 2)
    assert plan(W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=1), dvm.F64)[0] == "generic"
    assert plan(W.sod_1d(nx=200, nv=32, tau=1e-4), dvm.F32)[0] == "generic"
    with pytest.raises(dvm.DvmError):
        bad = W.sod_1d(nx=200, nv=32, tau=1e-4)
        cfg, keep = dvm.config_from_case(bad, precision=dvm.F32)
        cfg.grid.nx[0] = 0
        dvm.plan(cfg)
