"""GB300-native binary xyz interaction search (arXiv 1610.05108, Algorithm 2).

The search runs in hand-written sm_103a CUDA kernels behind a C ABI
(``include/xyz.h``); ``paper_1610_05108_gb300.xyz`` is the thin ctypes binding
and ``paper_1610_05108_gb300.synth`` makes seeded synthetic inputs.
"""
