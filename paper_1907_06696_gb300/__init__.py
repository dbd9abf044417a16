"""GB300 matrix-free GMG Stokes library (Clevenger & Heister, arXiv 1907.06696).

The compute path is the CUDA library libstokes_gb300.so (include/stokes.h);
`paper_1907_06696_gb300.capi` is its thin ctypes binding with the same entry
point names. Importing this package does not load the library.
"""
