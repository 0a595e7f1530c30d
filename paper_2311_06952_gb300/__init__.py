"""GB300-native hot path of MH-DEOCT (arXiv 2311.06952).

The compute lives in the C-ABI library ``libdeoct.so`` (hand-written CUDA for
sm_103a, declared in ``include/deoct.h``); ``paper_2311_06952_gb300.deoct`` is
its thin ctypes binding.  Importing this package does not load the library:
``datagen`` (seeded synthetic inputs) works without a GPU.
"""
__all__ = ["datagen", "deoct", "build"]
