"""GB300-native GP-FVM hot path: structured Gram matvec, Cholesky-deflated
CG/IterGP and posterior evaluation as hand-written sm_103a CUDA behind a C ABI
(include/gpfvm.h).  ``gpfvm`` is the ctypes binding; ``build`` compiles the
library in-tree."""
__all__ = ["gpfvm", "build"]
