"""GB300-native Strassen / Strassen-Winograd matrix product (arXiv 2309.00628).

The compute path is the C-ABI library ``libswmm.so`` (CUDA, sm_103a), declared in
``include/swmm.h``; :mod:`paper_2309_00628_gb300.swmm` is its thin ctypes binding.
"""
