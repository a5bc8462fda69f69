"""GB300-native agglomeration-based multigrid PCG for the SIPG-DG monodomain model.

The compute path lives in the CUDA/C++ library `libaggmg.so` (built from
`csrc/`); `aggmg` is its thin ctypes binding. `workloads` builds the seeded
synthetic inputs. Submodules are imported on demand so that importing the
input generators never loads the CUDA library.
"""
import importlib

__all__ = ["aggmg", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
