"""GB300-native phase-shift-dealiased pseudo-spectral Navier-Stokes step.

The compute path is the C-ABI library ``libns.so`` (hand-written sm_103a CUDA kernels,
declared in ``include/ns.h``); :mod:`paper_2603_08892_gb300.binding` is a thin ctypes
layer over it.  Importing this package does not load the library; ``binding`` does, and
fails loudly when it is missing.
"""

__all__ = ["binding", "inputs", "analysis"]
