"""GB300 (sm_103a) implementation of the COLA particle-mesh hot path (Koda et al. 2015, §2).

The compute lives in libcola.so (C ABI in include/cola.h); this package only builds it and
marshals torch tensors into it.  Importing the package does not load the library; the first
call that needs it does, and raises if it is missing.
"""

from .binding import Batch, ColaError, Context, Params, load_library, step_scalars  # noqa: F401
