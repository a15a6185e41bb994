"""GB300-native particle-mesh step for CDM and massive-neutrino particles.

The compute path is the C-ABI library ``libpmnu.so`` (hand-written sm_103a CUDA
kernels, declared in ``include/pm.h``); :mod:`paper_2007_13394_gb300.pm` is the
thin ctypes binding over it.  The library is loaded lazily on first use and a
missing or unloadable library raises an error: there is no CPU fallback.
"""
__all__ = ["inputs", "pm", "config"]
