"""GB300-native discrete-velocity BGK kinetic scheme (FKS/HOFKS of Dimarco & Loubere).

The compute path is the CUDA library ``libdvm.so`` behind the C ABI declared in
``include/dvm.h``; ``paper_1212_0204_gb300.dvm`` is its thin ctypes binding and is
imported on demand so that the input recipes in ``workloads`` load without a GPU.
"""
__all__ = ["dvm", "workloads"]
