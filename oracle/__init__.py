"""Oracle package: a plain FP64 CPU reference for element-local assembly.

Test infrastructure only.  The test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers; the CUDA library never imports it.
"""
from .oracle import *  # noqa: F401,F403
