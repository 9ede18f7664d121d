"""GB300 (sm_103a) lattice SIGW library: hot path of arXiv 2605.27231 behind a C ABI.

The compute path is libsigw.so (hand-written CUDA kernels, include/sigw.h);
``paper_2605_27231_gb300.sigw`` is its ctypes binding and ``build`` compiles it.
"""
