"""GB300 (sm_103a) plane-wave Bethe-Salpeter hot path behind a C ABI.

``bse`` is the ctypes binding of include/bse.h; ``pipeline`` chains the calls
into one forward pass.  Importing the package does not load the CUDA library;
``bse.load()`` does, and raises if it has not been built.
"""
