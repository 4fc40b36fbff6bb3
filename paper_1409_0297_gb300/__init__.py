"""GB300 (sm_103a) sparsifying-preconditioned GMRES for periodic Helmholtz and
Schroedinger problems (Ying, arXiv 1409.0297).

The compute lives in the CUDA library libsp_gb300.so (C ABI: include/sp.h);
`binding` is its ctypes binding.  Build the library with
`paper_1409_0297_gb300.build.build()`.  Importing `binding` fails if the
library is missing: there is no CPU path.
"""
__all__ = ["binding", "build"]
