"""FP64 CPU oracle for the Block CUR hot path.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.
"""
from .bcur_oracle import *  # noqa: F401,F403
