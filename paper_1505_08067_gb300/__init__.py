"""Batched complex FFT library for one GB300 (sm_103a).

The transforms run in hand-written CUDA kernels inside ``libgbfft.so``, reached
through its C ABI (``include/gbfft.h``).  ``gbfft`` is the thin Python binding
(argument marshalling only); ``synth`` makes seeded synthetic inputs.  Importing
the package loads nothing; the shared library is opened on first use and its
absence is an error, never a fallback.
"""
