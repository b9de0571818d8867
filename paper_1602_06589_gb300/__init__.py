"""GB300-native generation of the muffin-tin FLAPW Hamiltonian and overlap.

The compute path lives in a CUDA shared library (``csrc/``) behind a C ABI
(``include/hsgen.h``); ``hsgen`` is its thin ctypes binding.
"""
