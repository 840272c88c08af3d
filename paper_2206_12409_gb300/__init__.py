"""GB300-native hybrid volume-surface integral equation (hybrid-VSIE) library.

The compute path lives in the CUDA shared library ``libvsie`` (C ABI declared in
``include/vsie.h``); :mod:`paper_2206_12409_gb300.vsie` is the thin ctypes binding
and :mod:`paper_2206_12409_gb300.inputs` generates seeded synthetic workloads.
Nothing is loaded at import time.
"""
__all__ = ["inputs", "vsie"]
