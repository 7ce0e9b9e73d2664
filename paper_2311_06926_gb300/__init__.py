"""GB300 (sm_103a) hyper-power preconditioned Stokes solver (arXiv 2311.06926).

``Stokes`` wraps the C ABI of ``include/stokes_hp.h`` (CUDA library ``libstokes_hp.so``, built
by ``paper_2311_06926_gb300.build``). The library is loaded on first use, not at import.
"""
from .binding import Stokes, StokesError, load_library, LIB_PATH  # noqa: F401
