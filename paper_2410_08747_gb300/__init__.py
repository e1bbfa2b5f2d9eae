"""GB300-native forward Monte Carlo X-ray ray tracing (McXtrace-style hot path).

The traced path runs in hand-written sm_103a CUDA kernels behind a C ABI
(``include/mcx.h``); ``paper_2410_08747_gb300.mcx`` is the thin ctypes binding.
"""
