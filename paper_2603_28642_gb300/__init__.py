"""GB300-native row-splitting ILU preconditioned least squares.

The library (librlsq.so, built from csrc/ by ``build.build()``) implements
the hot path of Scott & Tuma's row-splitting ILU preconditioner inside LSMR
on one GPU; ``binding`` is its thin ctypes binding and ``synth`` the seeded
problem generators.  Submodules load lazily so that importing the package
does not require a GPU.
"""
__all__ = ["binding", "build", "synth"]


def __getattr__(name):
    import importlib

    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
