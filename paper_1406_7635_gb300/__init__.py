"""GB300-native finite-difference micromagnetics: effective field + adaptive RK45.

The compute path lives in ``csrc/`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/mm.h``); ``mm`` is the thin ctypes binding.
"""
