"""GB300-native (sm_103a) interval Mean Value Form subdomain bounding.

Subdomain Lower Bounding for spatial branch and bound (Zhang et al.,
"Accelerating Deterministic Global Optimization via GPU-parallel Interval
Arithmetic"): libivb.so (C ABI in include/ivb.h, CUDA kernels in csrc/) with a
thin ctypes binding (`ivb`), seeded synthetic workloads (`workloads`) and a
torch.autograd.Function for point gradients (`autograd`).

Submodules are imported lazily so that the input generator works on machines
without the CUDA library.
"""
import importlib

__all__ = ["ivb", "workloads", "build", "autograd", "shard"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
