"""FP64 CPU oracle of the well-balanced WCSPH step (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. It is a plain, slow, literal statement of the paper's
method in C (``wbsph_oracle.c``) behind a ctypes wrapper (``oracle.py``) and
shares no code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
