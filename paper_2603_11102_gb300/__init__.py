"""GB300-native (sm_103a) high-order gas-kinetic scheme step with ALM and IBM
forcing.

The compute path is the CUDA library ``libgks.so`` (hand-written kernels
behind a C ABI declared in ``include/gks_api.h``); ``gks`` is its thin ctypes
binding. ``workloads`` builds seeded synthetic inputs and needs no GPU.
Importing the package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "gks"]


def __getattr__(name):
    if name == "gks":
        import importlib
        return importlib.import_module(__name__ + ".gks")
    raise AttributeError(name)
