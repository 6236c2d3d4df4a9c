"""FP64 CPU oracle for the RGB-Depth-Normal Gaussian training step.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it.
"""
from .pgs_oracle import *  # noqa: F401,F403
