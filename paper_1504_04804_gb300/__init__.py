"""grx: GB300-native frontier graph traversal (arXiv 1504.04804's hot path).

Submodules:
  grx      -- ctypes binding of the C-ABI library libgrx.so (CUDA, sm_103a)
  inputs   -- seeded synthetic graphs, weights and sources
  serving  -- continuous-batching query server over resident graphs
  autotune -- per-graph search of the direction-switch and load-balance knobs
  build    -- compiles libgrx.so with nvcc

The binding is imported lazily so that ``inputs`` can be used on machines
without the compiled library; any traversal call without the library raises.
"""
import importlib

__all__ = ["grx", "inputs", "serving", "autotune", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
