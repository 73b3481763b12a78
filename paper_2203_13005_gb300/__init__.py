"""GB300-native GAS superstep engine (GX-Plug's daemon hot path, Section II-A and III).

The compute path lives in ``libgxp.so`` (CUDA for sm_103a behind the C-ABI
declared in ``include/gxp.h``); ``paper_2203_13005_gb300.gxp`` is the thin
ctypes binding to it and ``paper_2203_13005_gb300.synth`` the seeded input
generators. Importing the package loads nothing native: the binding loads
``libgxp.so`` on first use and raises if it is missing.
"""
__all__ = ["gxp", "synth", "build"]
