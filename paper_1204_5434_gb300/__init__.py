"""GB300-native pseudo-spectral propagator library for polymer field theory.

The compute path lives in the CUDA library ``libpft.so`` (C ABI: include/pft.h);
``paper_1204_5434_gb300.pft`` is its thin ctypes binding.  ``workloads`` draws the
seeded synthetic fields.
"""
from . import workloads  # noqa: F401

__all__ = ["pft", "workloads", "build"]
