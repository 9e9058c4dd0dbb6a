"""GB300-native FHP lattice gas (arXiv:1208.2428 hot path).

The update runs in hand-written CUDA for sm_103a behind the C ABI of
``include/fhp.h``; this package holds the CUDA sources (``csrc/``), their
build (``build.py``) and the ctypes binding (``fhp.py``).
"""
from .fhp import (SHAPE_DISC, SHAPE_ROWS, Batch, FhpError, Lattice, load, philox4x32_10_device,  # noqa: F401
                  required_bytes)

__all__ = ["Batch", "FhpError", "Lattice", "SHAPE_DISC", "SHAPE_ROWS", "load", "philox4x32_10_device",
           "required_bytes"]
