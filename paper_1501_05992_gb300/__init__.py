"""GB300 X-engine for the MWA correlator (4+4-bit FX cross-multiply-accumulate).

The CUDA library (``csrc/``, C ABI in ``include/corr.h``) holds every step of
the hot path; ``corr`` is its thin Python binding.  Importing this package
loads nothing: ``from paper_1501_05992_gb300 import corr`` loads the binding,
which loads (and if needed builds) ``_build/libcorr.so`` on first use.
"""
__all__ = ["corr", "build", "service"]
