"""GB300-native influence minimisation by node blocking (arXiv 2405.12871 hot path).

The library is the CUDA shared object built from ``csrc/`` (C ABI in
``include/imin.h``); ``_lib`` binds it with ctypes.  ``synth`` builds seeded
synthetic workloads.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "load"]


def load():
    """Import the ctypes binding (loads, and if needed builds, libimin.so)."""
    from . import _lib
    _lib.load()
    return _lib
