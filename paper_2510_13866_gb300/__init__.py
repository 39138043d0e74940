"""GB300 (sm_103a) worldline FFBS + Hirsch-Gibbs sampler for the 2D Hubbard model
(arXiv 2510.13866).  The compute path is the C-ABI library libhqmc.so built from csrc/;
this package is its Python binding."""
from .hqmc import HQMCError, Lattice, fp32_peak, fp64_peak, lib, log_weight, supported_L  # noqa: F401
