"""GB300-native exact-exchange (EXX) operator for free-boundary real-space grids.

The compute path is hand-written sm_103a CUDA behind the C ABI declared in
``include/exx.h``; :mod:`.exx` is a thin ctypes binding over it and
:mod:`.autograd` wraps it as a ``torch.autograd.Function``.  Submodules are
imported lazily so that the input generator (:mod:`.synth`) can be used
without loading the CUDA library.
"""

__all__ = ["exx", "autograd", "synth", "spin", "dist", "tune"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
