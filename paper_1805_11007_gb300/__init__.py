"""GB300-native particle step of the hybrid chemotaxis model of Bruna, Maini &
Robinson (arXiv:1805.11007): cell list, pair force, gradient interpolation,
Euler-Maruyama move, secretion deposit and chemical PDE, as hand-written CUDA
behind the C ABI declared in ``include/chemo.h``.

``paper_1805_11007_gb300.chemo`` is the ctypes binding of that library (the
same names as the C ABI). Importing the package itself loads nothing, so the
seeded input generators in ``workloads`` can be used without a GPU.
"""
import importlib

__all__ = ["chemo", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
