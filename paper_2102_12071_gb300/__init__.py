"""GB300-native learned-smoother multigrid (Huang, Li & Xi, arXiv 2102.12071).

The compute path lives in the CUDA library ``libmgcnn.so`` (sources under ``csrc/``,
C-ABI declared in ``include/mgcnn.h``); ``binding`` is its thin ctypes front end.
"""
