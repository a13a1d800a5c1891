"""Wavelet-domain l1-l2 deblurring on GB300 (Escande & Weiss, arXiv 1512.08401).

The compute path lives in the CUDA library ``libwdb.so`` built from ``csrc/``; ``wdb`` is
its ctypes binding (argument marshalling only). ``synthetic`` generates seeded inputs.
Importing this package does not load the library; ``wdb.lib()`` does, and raises if the
library has not been built.
"""
