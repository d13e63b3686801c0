"""GB300-native (sm_103a) taches-algorithm convolution.

The compute path is libtaches.so (CUDA kernels behind the C ABI of
include/taches.h). ``capi`` is its thin Python binding, with the same
entry-point names. ``synth`` holds the seeded synthetic workloads. Importing
this package loads nothing; the library loads on the first ``capi`` call and
raises if it has not been built.
"""
from . import capi, synth  # noqa: F401
from .capi import *  # noqa: F401,F403

__all__ = [n for n in dir(capi) if n.startswith("tc_")] + ["capi", "synth", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libtaches.so in-tree for sm_103a (nvcc)."""
    from . import _build
    return _build.build(force=force, verbose=verbose)
