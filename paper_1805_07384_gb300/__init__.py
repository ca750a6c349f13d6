"""Fixed-PSNR lossy compression for float32 fields on GB300 (sm_103a).

The compute path lives in the CUDA shared library built from ``csrc/``; the
Python side (``fpsnr.py``) only marshals arguments into its C ABI.  Importing
this package does not load the library; ``fpsnr.load()`` does, and fails
loudly if it has not been built.
"""
__all__ = ["fpsnr", "synth"]
