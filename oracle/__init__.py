"""FP64 CPU oracle for the diblock propagator path (test infrastructure only).

This package is test infrastructure.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library in ``paper_1204_5434_gb300`` and never imports it.
"""
from .pft_oracle import *  # noqa: F401,F403
from .philox import philox4x32_10, philox_normals  # noqa: F401
