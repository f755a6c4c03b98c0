"""GB300-native plasma-line spectrum integration (decode -> FFT -> |X|^2 over IPPs).

The compute path is the CUDA library ``lib/libisr.so`` behind the C ABI in
``include/isr.h``; ``isr`` is its thin Python binding.
"""
from . import isr  # noqa: F401
from .isr import Plan, IsrError  # noqa: F401

__all__ = ["isr", "Plan", "IsrError", "build"]


def build(force: bool = False, verbose: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force, verbose=verbose)
