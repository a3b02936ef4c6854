"""Evaluation points away from the start psi = 1 for the GPU parity tests.

With the free-space value ext = 1 the start point psi = 1 makes the object field
w = R0(psi - 1) vanish, so the bilinear gather of the object and the conj(w) v term of the
probe gradient contribute nothing there.  The parity tests therefore also evaluate at
  * the point after a few iterations of the oracle's own conjugate-gradient driver from
    the start point (small problems), and
  * the true object times a small complex perturbation (large problems, where the oracle's
    iterations would take minutes).
Both are rounded to complex64 so the GPU and the oracle see the same inputs.  Only the
oracle computes anything here; nothing comes from the CUDA path.
"""

import numpy as np

import holo_synth as hs
from oracle import cg as ocg


def c64(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


def iterated_point(psi0, q0, t, sqrt_d, sqrt_dref, geo, iters=5, probe_shifts=None):
    """(psi, q) after `iters` joint Dai-Yuan iterations of the oracle driver (Sec. 2, reading
    R7) from (psi0, q0); at most 8 step halvings per line search keep the cost small."""
    r = ocg.reconstruct(psi0, q0, t, sqrt_d, sqrt_dref, geo, iters, max_halvings=8,
                        probe_shifts=probe_shifts)
    return c64(r["psi"]), c64(r["q"])


def object_point(psi_true, rng, level=0.05):
    """The true object times 1 + level * complex standard normal noise."""
    return c64(hs.perturbed_probe(psi_true, rng, level))
