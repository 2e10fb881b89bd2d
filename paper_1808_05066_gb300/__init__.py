"""GB300 (sm_103a) implementation of the entropy-variable hybridized DG hot path:
per-element Newton linearisation and static condensation, trace solve, interior
recovery and BDF Newton steps (arXiv:1808.05066, Secs. 3.2-3.3).

The compute path is libhdg.so (CUDA, include/hdg.h); `hdg` is its ctypes binding.
Importing `paper_1808_05066_gb300.hdg` fails loudly if the library was not built.
"""
