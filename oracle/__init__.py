"""Plain FP64 CPU oracle for RQRCP / TRQRCP / TUXV (arXiv 2008.04447).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.
"""
from .rq_oracle import *  # noqa: F401,F403
