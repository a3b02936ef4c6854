"""GB300-native evaluation of the multi-distance holography functional with probe retrieval.

Nikitin et al., "X-ray nano-holotomography reconstruction with simultaneous probe
retrieval": the amplitude functional F2 (Eq. min1) or the intensity functional F1
(Eq. min2) and their gradients with respect to the per-angle transmittances psi_k and the
probe q (Eq. gradpsi), computed by hand-written sm_103a CUDA kernels behind the C ABI of
include/holo.h.

    from paper_2407_20304_gb300 import Holo
    h = Holo(n, n_angles, n_dist, wavelength, pixel, Z, z)
    h.set_shifts(t); h.set_data(sqrt_d, sqrt_dref); h.set_probe(q)
    loss, grad_psi, grad_q = h.gradient(psi)

Modules: holo (Holo, bin_amplitudes, upsample2), cg (the joint DY / FR / PRP conjugate
gradient driver with backtracking or Armijo line searches), hierarchy (reconstruction on
binned levels), batch (many reconstructions in one CUDA graph), autograd (a
torch.autograd.Function), dist (angle sharding over ranks).  The compiled library is built
in-tree by `paper_2407_20304_gb300.build.build()`.
"""

from .holo import Holo, bin_amplitudes, upsample2  # noqa: F401
from ._lib import HoloError, load  # noqa: F401

__all__ = ["Holo", "HoloError", "bin_amplitudes", "load", "upsample2"]
