"""GB300 (sm_103a) matrix-free DG solver for the acoustic wave equation.

Thin Python binding of the C ABI in include/dg.h (``libdg.so`` built in-tree
by ``build.py``).  Every step of the solver runs in the library's CUDA
kernels; this package only marshals arrays, pointers and streams.  Importing
it does not load the library; the first use does, and fails loudly if the
library is missing.
"""
from ._lib import (DGError, probe_fma_peak, Solver, Solver2D, Batch, Server, load_library, library_path,  # noqa: F401
                   DG_FP64, DG_FP32, EXPORTED_SYMBOLS, KIND_LSRK, KIND_ADER, KIND_TCK,
                   BASIS_GL, BASIS_G, PRED_AUTO, PRED_LINES, PRED_COLUMNS,
                   PRED_GL_PROJECTION, PRED_INTERLEAVED, LSRK_CK54, LSRK45, LSRK59)
