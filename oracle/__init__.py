"""FP64 CPU oracle for the IBMI block sweep.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The product path never
calls into it and shares no code with it.
"""
from .ibmi_oracle import *  # noqa: F401,F403
