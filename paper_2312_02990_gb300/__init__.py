"""GB300-native engine for the transient-time correlation function (TTCF)
method of arXiv:2312.02990: the ensemble of sheared daughter trajectories
spawned from the four mappings of equilibrium mother states.

The compute path is the CUDA library ``libttcf.so`` (sources in ``csrc/``,
C ABI in ``include/ttcf.h``); ``ttcf`` is a thin ctypes binding with the same
names.  Importing the package does not load the library; the first call that
needs it does, and raises if it is missing or no GPU is present.
"""
__all__ = ["ttcf", "inputs", "build"]
