"""GB300-native (sm_103a) NLOS transient simulator of arXiv 2506.03747.

The package holds the CUDA library sources (``csrc/``), its build script
(``build.py``) and the ctypes binding of the C ABI (``nlos.py``); the torch
autograd wrapper of the differentiable splat lives in ``autograd.py``.
Importing the package does not load the library; ``nlos.load()`` does, and
raises if ``libnlos.so`` has not been built (there is no CPU fallback).
"""
__all__ = ["nlos", "build"]
