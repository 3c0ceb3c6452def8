"""B300-native Plenoxel RGB-D render, grid adjoint and pose tracking.

The compute path lives in ``libplx.so`` (hand-written CUDA for sm_103a behind
the C ABI declared in ``include/plx.h``); ``plx`` is its ctypes binding and
``autograd`` wraps it for PyTorch. ``scenes`` holds the seeded input
generators. Importing this package does not load the CUDA library; importing
``paper_2307_03404_b300.plx`` does, and raises if it is missing.
"""
__all__ = ["scenes"]
