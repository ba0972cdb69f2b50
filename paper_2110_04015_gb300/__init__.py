"""GB300-native block-Jacobi PCG and multidirectional CG for the bundle-adjustment normal equation.

The compute path is the CUDA library ``libba`` (C ABI in ``include/ba.h``);
``binding`` is its ctypes binding and ``synthetic`` the seeded scene generator.
Importing the package loads nothing; ``binding.lib()`` loads the library and
raises if it is missing.
"""
