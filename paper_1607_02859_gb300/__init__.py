"""GB300-native hot path of the cubic-scaling space-time GW method.

The compute path lives in ``libgw.so`` (hand-written CUDA for sm_103a behind a
C ABI, see ``include/gw.h``).  ``paper_1607_02859_gb300.gw`` is the thin ctypes
binding; importing this package does not load the library.
"""
