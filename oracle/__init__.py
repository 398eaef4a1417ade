"""FP64 CPU oracle of the COLA particle-mesh method (Koda et al. 2015, arXiv:1507.05329).

TEST INFRASTRUCTURE ONLY.  Plain, slow numpy/scipy code in float64 that states what the
GPU path computes, one function per step of the method, each citing the passage of the
paper it follows.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import it.  The CUDA library shares no code, header, table or constant
generator with it, and it imports nothing from the CUDA package.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed forms,
invariants, brute force or values the mathematics fixes; none is pinned by re-running
itself.

Units: H0 = 1, lengths of the particle/mesh arrays in PM mesh cells (L / N), the time
variable is the scale factor a, velocities are canonical (v = a^2 dx/dt).
"""

from . import cosmology, cic, fourier, pm, lpt, power, cola, adjoint, fof, rng  # noqa: F401
from .cosmology import Params  # noqa: F401
