"""GB300-native SCF and MEX expansion force calculation (ETICS method).

The compute path is the CUDA library ``libetics.so`` (C ABI declared in
``include/etics.h``); :mod:`paper_1406_4254_gb300.etics` is its thin Python
binding.  The binding loads the library lazily, on first use, and raises if it
is missing: there is no CPU fallback.
"""
__all__ = ["etics", "inputs"]
