"""GB300-native (sm_103a) evaluation phase of the Empirical Interpolation FMM
(F. Casenave, arXiv:1408.0210).

The compute path is ``libeifmm.so`` (hand-written CUDA behind the C ABI of
``include/eifmm.h``); ``paper_1408_0210_gb300.eifmm`` is its thin ctypes
binding and ``paper_1408_0210_gb300.workloads`` draws the seeded synthetic
inputs.
"""
