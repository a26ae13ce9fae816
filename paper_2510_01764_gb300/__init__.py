"""GB300-native vectorised CHIP-8 environment step (Octax, arXiv 2510.01764).

``workloads`` (pure numpy input generators) imports nothing else; the CUDA
binding (``octax``) loads the in-tree ``liboctax.so`` on first use and raises if
it is missing: there is no CPU fallback.
"""
import importlib

__all__ = ["workloads", "octax", "Env"]


def __getattr__(name):
    if name == "Env":
        return importlib.import_module(__name__ + ".octax").Env
    raise AttributeError(name)
