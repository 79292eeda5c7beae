"""GB300-native structured LQ solver over 2D grids.

The compute path is the C-ABI library built from ``csrc/`` (CUDA for
sm_103a); ``lq2d`` is its thin ctypes binding.  ``synth`` draws seeded
synthetic problems and needs no GPU.
"""
import importlib

__all__ = ["lq2d", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
