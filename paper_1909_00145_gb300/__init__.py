"""GB300 (sm_103a) library for stochastic convolutional sparse coding.

The compute path is the CUDA shared library built from ``csrc/`` and exposed
through the C ABI declared in ``include/scsc.h``; :mod:`.scsc` is the thin
ctypes binding with the same names.  Importing this package loads nothing;
the library is loaded on first use and a missing library is an error.
"""

__all__ = ["scsc", "inputs", "build"]
