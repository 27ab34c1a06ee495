"""LeaFi oracle: TEST INFRASTRUCTURE ONLY.

A plain CPU restatement of the method (C library `leafi_oracle.c` + this ctypes
wrapper).  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it; the product path never does.
"""
from .oracle import *  # noqa: F401,F403
