"""pss: GB300-native per-DM-trial pulsar periodicity search.

The compute path lives in the CUDA shared library ``libpss.so`` (C ABI,
declared in ``include/pss.h``); ``paper_1912_12807_gb300.pss`` binds it with
ctypes.  ``synth`` makes seeded synthetic filterbanks.
"""
__all__ = ["synth", "pss"]
