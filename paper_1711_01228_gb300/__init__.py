"""GB300-native SOR stress-majorization graph layout (Wang & Wang, 2012).

The compute path is the CUDA library ``libfdlayout.so`` built from ``csrc/``
and called through its C ABI (``include/fd_layout.h``).  Importing the package
does not load the library; the first call into :mod:`.api` does, and fails
loudly if it is missing.  Submodules: ``api`` (the binding), ``synth`` (seeded
input generators), ``build`` (nvcc build of the library).
"""
