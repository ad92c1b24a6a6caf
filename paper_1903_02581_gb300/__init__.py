"""GB300-native split-step propagation of the two-electron Hong-Ou-Mandel wavefunction.

The compute path lives in the CUDA library ``libhom`` (``csrc/``), reached
through the C ABI declared in ``include/hom.h``; ``binding`` marshals
arguments to it.  Import of this package does not load the library: the
first call into ``binding`` does, and raises if it is missing.
"""
