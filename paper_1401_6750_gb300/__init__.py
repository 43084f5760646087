"""Truncated-solver disconnected fermion loops on one GB300 (sm_103a).

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python modules here only marshal arguments (``abi``), wrap the calls for
PyTorch tensors (``api``) and make seeded synthetic inputs (``synth``).
Importing the package does not load the library; ``abi.lib()`` does, and it
raises if the library has not been built.
"""
__all__ = ["abi", "api", "synth"]
