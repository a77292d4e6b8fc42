"""GB300 (sm_103a) per-shot material-gradient evaluation for time-domain elastic
full-waveform inversion in 3D PML-truncated media (arXiv:1504.08340).

The C ABI is declared in include/fwi.h and implemented by libfwi.so (CUDA);
this package is its Python binding. Loading fails loudly if the library has
not been built: there is no CPU path.
"""
from .fwi import EXPORTS, LIB_PATH, Context, FWIError, load_library  # noqa: F401

__all__ = ["Context", "FWIError", "load_library", "EXPORTS", "LIB_PATH"]
