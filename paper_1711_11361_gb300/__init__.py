"""GB300-native moving-boundary cut-cell sweeps (arXiv 1711.11361).

The compute path is the CUDA shared library built from ``csrc/`` and reached
through the C ABI declared in ``include/mb.h``; ``paper_1711_11361_gb300.mb``
is the thin ctypes binding over it.  ``inputs`` builds seeded problem
descriptions.  Importing this package does not load the library; importing
``paper_1711_11361_gb300.mb`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs"]
