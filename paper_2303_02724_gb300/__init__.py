"""GB300-native extremum-graph library (Morse decomposition + saddle-maximum arcs).

The computation runs in libeg.so (CUDA, sm_103a) behind the C ABI of
include/eg.h; ``eg`` is its Python binding and ``fields`` the seeded synthetic
inputs.
"""
from . import fields  # noqa: F401

__all__ = ["fields", "eg", "build"]


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)
