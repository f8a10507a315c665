"""GB300-native Power Variable Projection (PoVar) inner solve.

The compute path is the C-ABI CUDA library ``libpovar`` (hand-written kernels
for sm_103a); ``paper_2405_05079_gb300.povar`` is its thin ctypes binding.
Importing this package loads nothing: the library is opened on first use and
the binding raises if it has not been built.
"""
