"""GB300-native integration of very many independent ODE systems (one per GPU
thread) after Hegedus, arXiv:1810.03931.

The compute path is the CUDA library ``libodegpu.so`` (sources in ``csrc/``,
C ABI in ``include/odegpu.h``); ``odegpu`` is its thin Python binding.
"""
from . import odegpu  # noqa: F401
from .odegpu import ODEError  # noqa: F401

__all__ = ["odegpu", "ODEError"]
