"""FP64 CPU oracle for "Learning optimal multigrid smoothers via neural networks".

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package; the product path never does.
"""
from .oracle import *  # noqa: F401,F403
