"""GB300-native (sm_103a) next reaction random time algorithm (Liu & Wang, arXiv:2103.00405).

Submodules:
  workloads -- seeded synthetic networks and inputs (data only)
  _lib      -- ctypes binding of librandtime (include/randtime.h)
  api       -- Network, simulate, LogLik (torch tensors in, torch tensors out)
  build     -- nvcc build of librandtime.so
The CUDA library is loaded on first use of ``api``; nothing here falls back to the CPU.
"""
__all__ = ["workloads", "api", "build"]


def __getattr__(name):
    if name in ("api", "_lib", "build", "workloads", "autotune"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
