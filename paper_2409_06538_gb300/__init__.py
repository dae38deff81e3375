"""GB300 (sm_103a) Tensor Network Monte Carlo for the 2D +-J random-bond Ising model
(arXiv 2409.06538): boundary-MPS row environments, autoregressive whole-lattice proposals
and the Metropolis correction, behind the C ABI of include/tnmc.h (libtnmc.so)."""
from .buildlib import build, lib_path  # noqa: F401
from .server import TNMCServer  # noqa: F401
from .tnmc import (TNMC, TNMCPeriodic, couplings_pmj, disorder_average, env_build_occupancy,  # noqa: F401
                   nishimori_beta, torus_couplings_pmj)
