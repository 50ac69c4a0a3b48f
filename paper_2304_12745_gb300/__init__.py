"""GB300-native deep-unfolded PA-consumption precoder (arXiv 2304.12745).

The compute lives in ``libprecode.so`` (hand-written CUDA for sm_103a behind a
C ABI declared in ``include/precode.h``); ``capi`` is its ctypes binding and
``precoder.Plan`` a torch-facing wrapper.  ``channels`` draws seeded synthetic
inputs.  Importing ``capi`` or ``precoder`` requires the built library.
"""
__all__ = ["capi", "precoder", "channels"]
