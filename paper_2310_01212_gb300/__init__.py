"""LightKernel-GB300: persistent-thread work dispatch on one GPU (sm_103a).

The C ABI is include/lk.h; ``paper_2310_01212_gb300.lk`` binds it with the
same function names.  Importing this package loads nothing native; the first
binding call loads liblk.so (built by ``paper_2310_01212_gb300.build.build``)
and fails loudly if it is missing.
"""
from . import build  # noqa: F401

__all__ = ["build", "lk", "synth"]
