"""GB300 (sm_103a) augmented preconditioned CG with Krylov-subspace recycling (TRKS/SRKS).

The compute path is the CUDA library built from csrc/ (C ABI in include/krs.h); the
Python side is the ctypes binding in ``binding`` and the seeded workloads in
``problems``.  Importing the package does not load the library; ``binding.lib()`` does,
and raises if it cannot.
"""
__all__ = ["binding", "problems", "build"]
