"""GB300-native persistent-kernel (PERKS) solvers: stencils and CG.

Importing the package loads nothing native; the CUDA library is loaded on
first use of ``paper_2204_02064_gb300.api`` and raises if it is missing.
"""
__all__ = ["api", "inputs", "model"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
