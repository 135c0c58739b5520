"""GB300-native Flow Fields: dense correspondence-field search (arXiv 1508.05151).

The compute path is the CUDA library libflowfields.so (C ABI in
include/flowfields.h); ``ffapi`` is its thin Python binding and ``synth`` the
seeded synthetic pair generator.
"""
from . import _build

__all__ = ["build", "ffapi", "synth"]


def build(force=False):
    """Compile libflowfields.so for sm_103a in-tree and load it."""
    path = _build.build(force=force)
    from . import ffapi
    ffapi.lib()
    return path
