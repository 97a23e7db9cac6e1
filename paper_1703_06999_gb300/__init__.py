"""GB300-native vdW-DF nonlocal correlation (Roman-Perez--Soler FFT method).

The compute path lives in the CUDA library ``libvdwgb.so`` (sources in
``csrc/``, C-ABI in ``include/vdwgb.h``); :mod:`.binding` is a thin ctypes
layer over it.  :mod:`.inputs` makes seeded synthetic densities.
"""
__all__ = ["binding", "inputs"]
