"""FP64 CPU oracle of the EGLM-MHD block step (test infrastructure only).

Used by tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg.  The product
path never imports this package.
"""

from .oracle import Oracle, orc_params, orc_refine, flux, alpha, lf_flux, limiter, weno_faces, prolong_1d, block_step

__all__ = ["Oracle", "orc_params", "orc_refine", "flux", "alpha", "lf_flux", "limiter",
           "weno_faces", "prolong_1d", "block_step"]
