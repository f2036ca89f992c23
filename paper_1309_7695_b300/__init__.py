"""B300-native batched stochastic simulation (tau-leaping with exact-SSA
fallback) of mass-action reaction networks.

The compute path is the CUDA library ``libtauleap.so`` behind a C ABI
(``include/tauleap.h``); :mod:`paper_1309_7695_b300.abi` is its thin Python
binding and :mod:`paper_1309_7695_b300.inputs` generates seeded synthetic
workloads.
"""
