"""LapH meson/baryon block contraction on GB300 (sm_103a).

The compute path is the C-ABI CUDA library in ``csrc/`` (declared in
``include/laph.h``); ``binding`` is a thin ctypes layer over it.  Importing
this package does not load the library; the first call into ``binding``
does, and raises if the library has not been built.
"""
import importlib

from . import synth  # noqa: F401

__all__ = ["synth", "binding"]


def __getattr__(name):
    if name == "binding":
        return importlib.import_module(__name__ + ".binding")
    raise AttributeError(name)
