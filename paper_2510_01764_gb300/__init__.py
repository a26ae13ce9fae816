"""GB300-native vectorised CHIP-8 environment step (Octax, arXiv 2510.01764).

``workloads`` (pure numpy input generators) imports nothing else; the CUDA
binding (``octax``) loads the in-tree ``liboctax.so`` on first use and raises if
it is missing: there is no CPU fallback.
"""
__all__ = ["workloads", "octax"]


def __getattr__(name):
    if name in ("octax", "Env", "Server"):
        from . import octax as _o
        return _o if name == "octax" else getattr(_o, name)
    raise AttributeError(name)
