"""Enforced-sparsity ALS NMF (arXiv:1510.05237) on GB300 (sm_103a).

The computation lives in the CUDA library built from ``csrc/`` (C ABI:
``include/espnmf.h``); ``binding`` marshals arguments to it.  Importing this
package does not load the library; the first call does, and raises if the
library has not been built.
"""
from .binding import *  # noqa: F401,F403
from .binding import (Context, EspnmfError, load, library_path,  # noqa: F401
                      exported_symbols)
