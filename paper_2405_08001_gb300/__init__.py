"""GB300-native (sm_103a) PNCG solver for interior-point Neo-Hookean elastodynamics (Shen et al., SIGGRAPH 2024).

The solver lives in a CUDA shared library behind a C ABI (``include/pncg.h``); ``binding`` wraps it with ctypes.
``scenes`` builds seeded synthetic inputs.  Importing this package does not load the library.
"""
