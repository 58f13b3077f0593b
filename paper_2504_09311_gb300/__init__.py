"""GB300-native batch peeling for densest-subgraph discovery (Dupin, arXiv 2504.09311).

The compute path is ``libdupin.so`` (hand-written sm_103a CUDA behind the C ABI in
``include/dupin.h``); ``dupin`` is its thin ctypes binding and ``synth`` the
seeded input generator.
"""
__version__ = "0.1.0"
