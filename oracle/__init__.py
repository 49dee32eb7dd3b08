"""FP64 CPU oracle for Richardson-Lucy and scaled gradient projection (SGP) deconvolution.

Test infrastructure: only the test-suite, the smoke check and the benchmark's CPU-baseline leg
use this package.  The CUDA product path never imports it.
"""
from .sgp_oracle import *  # noqa: F401,F403
