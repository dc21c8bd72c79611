"""GB300-native parallel cellular Potts model sweep.

The compute path is the CUDA library ``libcpm_gb300.so`` (sources in
``csrc/``, C ABI in ``include/cpm.h``); ``cpm`` is its Python binding.
"""
from . import build  # noqa: F401

__all__ = ["build", "cpm"]
