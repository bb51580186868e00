"""GB300-native staggered phase-field fracture solver (arXiv 2209.07969).

The solver is the CUDA library ``libpf`` (C ABI in ``include/pf.h``); ``binding``
loads it with ctypes.  ``specimens`` builds synthetic inputs.  Importing this package
does not load the library; ``binding.lib()`` does, and raises if it is missing.
"""
