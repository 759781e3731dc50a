"""FP64 CPU oracle for the image-plane single-pulse search (test infrastructure).

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg use
this package.  It shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
