"""CPU oracle (test infrastructure only): the plain double-precision
definition of the structured LQ solve that the CUDA path is checked against.
Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package."""
from .lq2d_oracle import *  # noqa: F401,F403
