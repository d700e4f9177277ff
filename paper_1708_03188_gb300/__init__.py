"""GB300-native spectral Galerkin hot path (Shenfun, arXiv 1708.03188).

Submodules are imported on demand so that ``inputs`` (seeded synthetic data)
can be used without loading the CUDA library:
  sgm      ctypes binding of the C-ABI library ``libsgm.so`` (the product path)
  inputs   seeded synthetic inputs and manufactured solutions
  build    nvcc build of ``libsgm.so`` for sm_103a
"""
import importlib

__all__ = ["sgm", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
