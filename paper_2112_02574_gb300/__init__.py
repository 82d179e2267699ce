"""GB300-native two-component Shan-Chen lattice Boltzmann (arXiv:2112.02574).

The compute path is the CUDA library ``_lib/libscgb.so`` (C ABI in
include/sc.h); ``binding`` marshals arguments to it with ctypes and PyTorch
device memory.  ``build`` compiles the library in-tree.
"""
import importlib

from .build import build  # noqa: F401

__all__ = ["build", "binding"]


def __getattr__(name):
    if name == "binding":
        return importlib.import_module(".binding", __name__)
    raise AttributeError(name)
