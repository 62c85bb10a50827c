"""GB300-native implicit Stokes step of the DLM level-set wave-structure
interaction method (Nangia, Patankar & Bhalla, arXiv 1901.07892).

The compute path is the CUDA library ``libwsi.so`` (sources in ``csrc/``,
C ABI in ``include/wsi.h``); ``wsi`` is its thin ctypes binding.  Importing
the package does not load the library; ``wsi.lib()`` does, and raises if it
is missing.
"""
