"""GB300-native forward/adjoint vector spherical harmonic transforms (FaVeST,
arXiv 1908.00041) on Gauss-Legendre grids.

The compute path is the CUDA library ``libfavest.so`` (C ABI in ``include/favest.h``);
``api`` is a thin ctypes binding with the same entry-point names, ``autograd`` wraps
the transforms as ``torch.autograd.Function``.  Importing this package does not load
the library; the first call into ``api`` does, and raises if it is missing.
"""
import importlib

__all__ = ["api", "autograd", "synthetic", "build"]


def __getattr__(name):
    if name in ("api", "autograd", "synthetic", "build"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
