"""FINOM on GB300: fast Sinkhorn for the entropic W1 distance on non-uniform meshes.

The computation lives in ``libfinom.so`` (hand-written sm_103a CUDA, C ABI in
``include/finom.h``); ``api`` is its thin Python binding and ``inputs`` the
seeded workload generators.  Importing the package does not load the library;
``api.load()`` (or the first call) does, and raises if it is missing.
"""
__all__ = ["api", "inputs", "build"]
