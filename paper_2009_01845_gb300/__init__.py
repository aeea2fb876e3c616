"""GB300-native state-vector quantum simulator core (Qibo, arXiv:2009.01845).

The compute path is the CUDA library ``libqsim_gb300.so`` built from
``csrc/`` for sm_103a; ``qsim`` is a thin ctypes binding over its C-ABI
(``include/qsim.h``). ``inputs`` generates seeded synthetic workloads and
holds none of the simulator's arithmetic. Importing this package loads nothing;
the library is opened on first use and a missing build raises at that point.
"""
__all__ = ["inputs"]
