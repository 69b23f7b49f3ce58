"""GB300 (sm_103a) Jacobian-free Newton-GMRES with the DG->FV multigrid
preconditioner of Birken, Dedner, Kloefkorn (arXiv 2505.24504).

The compute path is libjfnk.so (hand-written CUDA behind the C ABI of
include/jfnk.h); `jfnk` is a ctypes binding with the same names.  There is no
CPU path: without the built library or a CUDA device the calls raise.
"""
from .jfnk import (Batch, Context, Grid, JfnkError, Opts, Physics, Stats, lib, lib_path)  # noqa: F401

__all__ = ["Batch", "Context", "Grid", "Opts", "Physics", "Stats", "JfnkError", "lib", "lib_path"]
