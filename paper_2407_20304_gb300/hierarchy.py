"""Hierarchical reconstruction (Sec. 3, on speeding up the method): CG iterations on binned
data, then the recovered object and probe extrapolated to a grid twice as dense as the start
of the next, less binned level, ending without binning.

Level (b, iters): data binned by b (amplitudes sqrt of the b x b mean intensity,
holo_bin_amplitudes), pixel b dx, psi side n/b on a P/b grid, shifts t/b (and probe shifts
s/b when given), `iters` iterations
of the joint psi / q driver (cg.Reconstruction).  The first level starts from psi = 1 and the
paper's initial probe (the binned reference image propagated back to plane 0); later levels
start from the previous level's psi and q upsampled (holo_upsample2).  The FP64 oracle's
reconstruct_hierarchical takes the same steps.
"""

import numpy as np

from .cg import Reconstruction
from .holo import Holo, bin_amplitudes, upsample2


class Hierarchy:
    def __init__(self, n, n_angles, n_dist, wavelength, pixel, Z, z, shifts, pad=0,
                 levels=((8, 1000), (4, 500), (2, 250), (1, 125)), probe_shifts=None, **driver):
        P = pad or 2 * n
        bs = [b for b, _ in levels]
        if bs[-1] != 1 or any(bs[i] != 2 * bs[i + 1] for i in range(len(bs) - 1)):
            raise ValueError("binnings must halve from level to level and end at 1")
        if n % bs[0] or P % bs[0]:
            raise ValueError("n and the pad must be divisible by the coarsest binning")
        self.geo = dict(n=n, P=P, n_angles=n_angles, n_dist=n_dist, wavelength=wavelength,
                        pixel=pixel, Z=Z, z=tuple(z))
        self.shifts = np.asarray(shifts, np.float32)
        self.probe_shifts = None if probe_shifts is None else np.asarray(probe_shifts, np.float32)
        self.levels = tuple(levels)
        self.driver = driver
        self.results = []

    def run(self, sqrt_d, sqrt_dref, q0=None, callback=None):
        """sqrt_d [K][J][n][n], sqrt_dref [n][n]: float32 CUDA amplitudes.  Returns (psi, q) on
        the full grid; per-level histories are in self.results."""
        import torch
        g = self.geo
        psi = q = None
        for i, (b, iters) in enumerate(self.levels):
            nb, Pb = g["n"] // b, g["P"] // b
            h = Holo(nb, g["n_angles"], g["n_dist"], g["wavelength"], g["pixel"] * b, g["Z"],
                     g["z"], pad=Pb)
            if self.probe_shifts is not None:
                h.set_probe_shifts(np.ascontiguousarray(self.probe_shifts / b))
            h.set_shifts(np.ascontiguousarray(self.shifts / b))
            d = bin_amplitudes(sqrt_d, b) if b > 1 else sqrt_d
            dr = bin_amplitudes(sqrt_dref, b) if b > 1 else sqrt_dref
            h.set_data(d.contiguous(), dr.contiguous())
            if i == 0:
                psi = torch.ones((sqrt_d.shape[0], nb, nb), dtype=torch.complex64,
                                 device=sqrt_d.device)
                q = h.initial_probe(dr.contiguous()) if q0 is None else q0
            else:
                psi, q = upsample2(psi), upsample2(q)
            rec = Reconstruction(h, psi, q, **self.driver)
            rec.run(iters)
            psi, q = rec.psi, rec.q
            self.results.append({"b": b, "history": rec.history})
            if callback:
                callback(b, rec)
            h.close()
        return psi, q
