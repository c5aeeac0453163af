"""CPU checks of the boundary: libdvm.so builds, loads without a GPU and exports
every function include/dvm.h declares; the binding's list agrees with the header.
No compute call is made here."""
import ctypes
import os
import re

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
