"""GB300-native multiple-precision Taylor integrator for the Lorenz system.

Hot path of Dimova et al., "OpenMP parallelization of multiple precision
Taylor series method" (arXiv 1908.09301): Eq. (3)'s coefficient recursion with
exact Cauchy sums over L-limb numbers, division by (i+1), and Eq. (2) by
Horner's rule, in hand-written sm_103a kernels behind the C ABI of
``include/mpt.h``.  ``mpt`` is the thin ctypes binding.
"""

__all__ = ["mpt", "workloads", "build"]
