"""GB300 (sm_103a) deflated Arnoldi approximation of sgn(H_w(mu)) b.

Bloch, Wettig, Frommer, Lang, "An iterative method to compute the overlap
Dirac operator at nonzero chemical potential" (arXiv:0710.0341).

The computation lives in the CUDA library ``libovl.so`` (C ABI in
``include/ovl.h``); ``paper_0710_0341_gb300.ovl`` is its ctypes binding.
Importing this package does not load the library; ``ovl.lib()`` does, and
raises if it has not been built (``paper_0710_0341_gb300.build.build()``).
"""
__version__ = "0.1.0"
