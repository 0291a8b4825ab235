"""B300-native Spectral Ewald far-field grand mobility (Wang & Brady, arXiv 1506.08481).

The compute path is the CUDA shared library built from ``csrc/`` (C ABI declared
in ``include/se_mobility.h``); ``api`` is a thin ctypes binding over it.
Importing the package does not load the library; ``api.load()`` does, and
raises if the library is missing.
"""
