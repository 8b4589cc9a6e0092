"""B300 (sm_103a) implementation of the LPC3D lattice-propagation hot path.

The per-step stencil of the lattice-gas / moment-propagation model of
arXiv 2603.22553 (population hops with Metropolis weights, magnetisation
rotation, FID / population / MSD reductions) runs in hand-written CUDA
kernels behind the C ABI of ``include/lpc3d.h``; this package is the thin
Python binding (``binding``), a handle class (``lattice.Lattice``), the
downstream analysis (``downstream``) and the serving loop (``serve``).
"""
from .binding import LPCError, load  # noqa: F401

__all__ = ["LPCError", "load"]
