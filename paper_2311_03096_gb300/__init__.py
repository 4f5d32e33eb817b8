"""GB300-native proximal map of the weight-sharing penalty (arXiv 2311.03096).

The compute path lives in ``libws_prox.so`` (hand-written sm_103a CUDA behind a
C ABI, see ``include/ws_prox.h``); ``paper_2311_03096_gb300.ws`` is the thin
ctypes binding over it.  Importing this package loads nothing: the binding
loads the library on first use and raises if it is missing.
"""
