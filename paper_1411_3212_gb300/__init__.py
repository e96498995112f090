"""GB300-native repeated range queries over moving objects.

The compute path is libmqr.so (hand-written CUDA for sm_103a behind the C ABI
of include/mqr.h); ``paper_1411_3212_gb300.mqr`` is its ctypes binding and
``paper_1411_3212_gb300.workloads`` draws seeded synthetic inputs.
"""
