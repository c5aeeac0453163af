"""Host-side logic of bench.py that needs no GPU: the clock/throttle summary of the
nvidia-smi samples, the DRAM-traffic record keyed by the kernel sources, the bounded
oracle sample of the CPU baseline, the GPU index under CUDA_VISIBLE_DEVICES and the
roofline peak."""
import json
import os

import numpy as np

import bench
from paper_1212_0204_gb300 import workloads as W


def test_clock_summary_takes_median_max_and_active_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "2070, 2070, Not Active, Not Active, Not Active, Not Active",
        "2040, 2070, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "1980, 2070, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


def test_recorded_traffic_only_for_the_current_kernel_source(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "kinetic_pass_traffic.txt").write_text(
        "# comment line\n"
        "workload=quadrant_2d source=aaaaaaaaaaaaaaaa dram_bytes_per_launch=495203584\n"
        "workload=density_wave_3d_64 source=bbbbbbbbbbbbbbbb dram_bytes_per_launch=28584552448\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kinetic_source_hash", lambda: "aaaaaaaaaaaaaaaa")
    assert bench.recorded_traffic("quadrant_2d") == 495203584.0
    assert bench.recorded_traffic("density_wave_3d_64") is None  # taken on other sources
    assert bench.recorded_traffic("no_such_workload") is None


def test_kinetic_source_hash_covers_the_kernel_sources():
    h = bench.kinetic_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    # every source of the kinetic-pass kernels enters the key
    import inspect
    src = inspect.getsource(bench.kinetic_source_hash)
    csrc = os.path.join(os.path.dirname(bench.__file__), "paper_1212_0204_gb300", "csrc")
    for f in ("dvm_kinetic.cu", "dvm_kinetic_shapes.cu", "dvm_window_kernel.cuh", "dvm_window.cuh",
              "dvm_tile_kernel.cuh", "dvm_linmom.cu"):
        assert os.path.exists(os.path.join(csrc, f)) and f in src


def test_oracle_sample_is_bounded_and_keeps_the_velocity_grid():
    case = W.quadrant_2d(n=256, nv=32, tau=1e-3, steps=500)
    cases, what = bench.oracle_sample(case, 4e6)
    (c,) = cases
    assert c.nv == case.nv and c.dv == case.dv and c.tau == case.tau
    assert c.points <= 1.1 * 4e6 and c.nx[0] < 256 and "cells" in what
    tubes = W.batched_tubes(ncases=64, steps=2)
    picked, what = bench.oracle_sample(tubes, 1e6)
    pts = sum(t.points for t in picked)
    assert picked == tubes[:len(picked)] and pts >= 1e6 and pts - picked[-1].points < 1e6


def test_physical_gpu_index_follows_visible_devices(monkeypatch):
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,3")
    assert bench.physical_gpu_index(0) == 5 and bench.physical_gpu_index(1) == 3
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.physical_gpu_index(2) == 2


def test_peak_is_the_measured_copy_bandwidth(monkeypatch, tmp_path):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6769.4, "bf16_tflops": 1900.0}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, kind = bench.load_peaks()
    assert np.isclose(peak, 6769.4) and kind == "measured"
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    assert bench.load_peaks() == (6800.0, "fallback")


class _FakeSolver:
    """Stand-in for dvm.Solver on the CPU: advances with the oracle and adds a
    planted relative error `eps` to the density row."""
    eps = 0.0

    def __init__(self, case):
        import oracle
        from tests.helpers import grid
        self.o = oracle.Scheme(grid(case), tau=case.tau)

    @classmethod
    def from_case(cls, case, precision=None):
        return cls(case)

    def set_moments(self, U):
        self.o.set_moments(U)

    def step(self, n):
        self.o.step(n)

    def moments(self):
        U = self.o.moments()
        U[0] *= 1.0 + self.eps
        return U

    def f(self):
        return self.o.f() * (1.0 + self.eps)

    def kinetic_kernel(self):
        return "fake"

    def close(self):
        pass


class _FakeDvm:
    Solver = _FakeSolver


def test_precision_error_reports_the_moment_error_against_the_oracle():
    case = W.quadrant_2d(n=256, nv=16, tau=1e-3, steps=500)
    sample, what = bench.oracle_sample(case, 2e5)
    _FakeSolver.eps = 0.0
    r = bench.precision_error(_FakeDvm, sample, None, batch=False)
    assert r["max_rel_moment_err"] == 0.0 and r["max_rel_f_err"] == 0.0
    assert r["kinetic_kernel"] == "fake" and r["steps"] == 2
    _FakeSolver.eps = 3e-6
    r = bench.precision_error(_FakeDvm, sample, None, batch=False)
    assert np.isclose(r["max_rel_moment_err"], 3e-6, rtol=1e-6)
    assert np.isclose(r["max_rel_f_err"], 3e-6, rtol=1e-6)


def test_moment_error_scales_rows_by_density():
    Uo = np.array([[1.0, 2.0], [1e-9, -1e-9], [3.0, 3.0]])
    Ug = Uo.copy()
    Ug[1, 0] += 1e-6  # a near-zero momentum row is measured against |rho|_inf = 2
    assert np.isclose(bench.moment_err(Ug, Uo), 5e-7)


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args,
                          cwd=bench.ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference: the untuned FP64 oracle on the host, one JSON line with
    the arm's metric and unit, at least 3 warm-up steps, and cpu_baseline / e2e
    describing the same run (no host-device copies)."""
    r = _run_bench(["--impl", "reference", "--workload", "sod_1d", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT,
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_bench(["--impl", "reference", "--workload", "sod_1d", "--steps", "2"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""
