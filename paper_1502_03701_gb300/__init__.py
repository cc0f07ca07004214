"""GB300-native matrix-free global stability analysis of compressible flows.

The computation lives in the CUDA library ``libstab.so`` (C ABI in
include/stab.h); this package is its ctypes binding plus the in-tree build.
"""
from .binding import (EigResult, JvBatch, Server, Stab, StabError, default_opts, eigs_batch,  # noqa: F401
                      estimate_bytes, load)
