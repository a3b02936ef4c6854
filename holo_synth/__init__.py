"""Seeded synthetic inputs for the holography workloads.

Phantom transmittances psi_k, the striped probe q, the sample shifts t_kj, Poisson
counting noise and the instrument geometries.  Both the FP64 oracle tests and the GPU
library's tests / benchmark draw their inputs here.  This module holds none of the
method's arithmetic: no propagation, no resampling, no functional or gradient.
Noise is applied to intensities that the caller computed.

The paper's own phantom (an ALD-like cube, Sec. 3) and its near-field-ptychography
probe are not available; these generators stand in for them with the paper's shapes:
a layered cube projected at angles in [0, pi), a Gaussian probe with horizontal and
vertical stripes of a few pixels' period (the multilayer-mirror features of Fig. 1 and
Fig. 3), random sub-pixel sample shifts, and Poisson noise.
"""

import json
import os
from dataclasses import dataclass

import numpy as np

SEED_BASE = 240720304

# The synthetic configurations 0 .. 4 (tiny, medium, autograd, batch, large), their geometry
# and flags, as data: configs.json next to this file.
CONFIG_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")
_CONFIGS = json.load(open(CONFIG_PATH))

# Geometry of the synthetic workloads: lambda = 3.72e-11 m, 10 nm object-plane pixel,
# focus-to-sample distances z_j and focus-to-detector distance Z of Table 1.
WORKLOAD_GEOMETRY = {
    "wavelength": _CONFIGS["geometry"]["wavelength"],
    "pixel": _CONFIGS["geometry"]["pixel"],
    "Z": _CONFIGS["geometry"]["Z"],
    "z": tuple(_CONFIGS["geometry"]["z"]),
}

# The paper's instrument (Table 1): 17.05 keV, Z = 1.208 m, z_j in mm.
PAPER_GEOMETRY = {
    "wavelength": 7.27183e-11,
    "pixel": 1.0e-8,
    "Z": 1.208,
    "z": (4.026e-3, 4.199e-3, 4.890e-3, 6.325e-3),
}


@dataclass(frozen=True)
class Workload:
    """One synthetic reconstruction problem (sizes, generator choices, seed)."""

    name: str
    n: int
    P: int
    n_angles: int
    n_dist: int
    phantom: str          # "ellipses" or "layers"
    probe_sigma: float    # Gaussian sigma of the probe amplitude, pixels
    counts: float         # mean Poisson counts per pixel (0 = noiseless)
    chunk: int            # angles per gradient evaluation
    seed: int


def config(which):
    """Configuration `which` (index 0 .. 4 or name) of configs.json, as a dict; its seed is
    SEED_BASE + seed_offset."""
    for c in _CONFIGS["problems"]:
        if which in (c["index"], c["name"]):
            return dict(c, seed=SEED_BASE + c["seed_offset"])
    raise KeyError(which)


def holo_geometry(which, chunk=None):
    """The fields of the library's holo_geometry for a single-problem configuration (n, pad,
    n_angles, n_dist, chunk, wavelength, pixel, Z, z, w_ref, ext)."""
    c = config(which)
    if isinstance(c["pad"], str):
        raise ValueError(f"configuration {c['name']} has no single geometry")
    g = _CONFIGS["geometry"]
    f = _CONFIGS["flags"]
    return {"n": c["n"], "pad": c["pad"], "n_angles": c["n_angles"], "n_dist": c["n_dist"],
            "chunk": c["chunk"] if chunk is None else chunk, "wavelength": g["wavelength"],
            "pixel": g["pixel"], "Z": g["Z"], "z": list(g["z"][:c["n_dist"]]),
            "w_ref": f["w_ref"], "ext": f["ext"]}


def workloads():
    """The single-problem synthetic workloads of configs.json: tiny, medium, autograd-sized,
    large (the batch, configuration 3, is a list of problems drawn from its ranges)."""
    out = {}
    for c in _CONFIGS["problems"]:
        if isinstance(c["pad"], str):
            continue
        out[c["name"]] = Workload(c["name"], c["n"], c["pad"], c["n_angles"], c["n_dist"],
                                  c["phantom"], c["probe_sigma"], c["counts"], c["chunk"],
                                  SEED_BASE + c["seed_offset"])
    return out


def rng_for(seed, stream=0):
    """Independent PCG64 stream `stream` of a workload seed."""
    return np.random.Generator(np.random.PCG64([seed, stream]))


def transmittance(phase, absorption_ratio=50.0):
    """psi = exp(i phi + phi / ratio): phase phi <= 0 with absorption beta = delta / ratio."""
    phase = np.asarray(phase, dtype=np.float64)
    return np.exp(1j * phase + phase / absorption_ratio)


def ellipse_phase(n, rng, count=6):
    """Phase map of `count` random ellipses painted in order (later ones overwrite).

    Phase U(-1, 0) rad, centres in the central 60 %, semi-axes U(n/16, n/4),
    orientation U(0, pi).
    """
    yy, xx = np.meshgrid(np.arange(n) - n / 2, np.arange(n) - n / 2, indexing="ij")
    phase = np.zeros((n, n))
    for _ in range(count):
        val = rng.uniform(-1.0, 0.0)
        cy, cx = rng.uniform(-0.3 * n, 0.3 * n, size=2)
        ay, ax = rng.uniform(n / 16, n / 4, size=2)
        th = rng.uniform(0.0, np.pi)
        c, s = np.cos(th), np.sin(th)
        u = (xx - cx) * c + (yy - cy) * s
        v = -(xx - cx) * s + (yy - cy) * c
        phase[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] = val
    return phase


def _cube_chord(h, offsets, theta):
    """Path length through the square [-h, h]^2 of a ray at angle theta, per offset."""
    d = np.array([np.cos(theta), np.sin(theta)])
    nrm = np.array([-d[1], d[0]])
    lo = np.full(offsets.shape, -np.inf)
    hi = np.full(offsets.shape, np.inf)
    for ax in range(2):
        p0 = offsets * nrm[ax]
        if abs(d[ax]) < 1e-12:
            inside = np.abs(p0) <= h
            lo = np.where(inside, lo, np.inf)
            continue
        a = (-h - p0) / d[ax]
        b = (h - p0) / d[ax]
        lo = np.maximum(lo, np.minimum(a, b))
        hi = np.minimum(hi, np.maximum(a, b))
    return np.maximum(hi - lo, 0.0)


class LayeredCube:
    """A centred cube of 30 nested cubic shells (ALD-standard-like, Sec. 3 and Sec. 4).

    Shell thicknesses U{2..20} px, per-shell phase density U(0.05, 0.3) rad per pixel
    of path, shells alternating between the two materials' densities.  Projections are
    taken about the vertical axis at theta_k = pi k / N_theta and scaled so that the
    deepest projected phase is -pi at theta = pi/4.
    """

    def __init__(self, n, rng, layers=30, size_frac=0.6):
        self.n = n
        half = size_frac * n / 2
        hs, dens = [], []
        h = half
        mat = rng.uniform(0.05, 0.3, size=2)
        for i in range(layers):
            if h <= 0.5:
                break
            hs.append(h)
            dens.append(mat[i % 2] * rng.uniform(0.8, 1.2))
            h -= rng.integers(2, 21)
        self.h = np.array(hs)
        self.density = np.array(dens)
        # shell i occupies cube(h_i) minus cube(h_{i+1}), so the projected phase is
        # -sum_i rho_i (proj(h_i) - proj(h_{i+1})) = -sum_i (rho_i - rho_{i-1}) proj(h_i)
        self.coef = self.density - np.concatenate(([0.0], self.density[:-1]))
        self.scale = 1.0
        self.scale = np.pi / max(1e-12, -self.phase(np.pi / 4).min())

    def phase(self, theta):
        """Projected phase (<= 0) of the cube at rotation angle theta: n x n."""
        off = np.arange(self.n) - self.n / 2 + 0.5
        A = np.stack([_cube_chord(h, off, theta) for h in self.h], axis=1)     # [x][l]
        B = (np.abs(off)[:, None] <= self.h[None, :]).astype(np.float64)      # [y][l]
        return -self.scale * (B * self.coef[None, :]) @ A.T


def object_stack(workload, angles, rng):
    """psi_k for the given angle indices of a workload: [len(angles)][n][n] complex128."""
    n = workload.n
    if workload.phantom == "ellipses":
        return np.stack([transmittance(ellipse_phase(n, rng)) for _ in angles])
    cube = LayeredCube(n, rng)
    return np.stack([transmittance(cube.phase(np.pi * k / workload.n_angles)) for k in angles])


def striped_probe(P, sigma, rng, stripes=6, strength=0.2, phase_amp=0.5):
    """Probe on the P x P grid: Gaussian amplitude (sigma px) times 1 + strength *
    sum of `stripes` horizontal/vertical sinusoids of period U(3, 12) px, with a stripe
    phase of amplitude `phase_amp` rad built the same way (mean of `stripes` sinusoids).
    A negative amplitude factor is kept as is (a phase of pi)."""
    c = np.arange(P) - P / 2
    yy, xx = np.meshgrid(c, c, indexing="ij")

    def stripe_sum():
        acc = np.zeros((P, P))
        for _ in range(stripes):
            period = rng.uniform(3.0, 12.0)
            ph = rng.uniform(0.0, 2.0 * np.pi)
            coord = yy if rng.integers(0, 2) == 0 else xx
            acc += np.sin(2.0 * np.pi * coord / period + ph)
        return acc

    amp = np.exp(-(xx ** 2 + yy ** 2) / (2.0 * sigma ** 2)) * (1.0 + strength * stripe_sum())
    phase = phase_amp * stripe_sum() / stripes
    return amp * np.exp(1j * phase)


def sample_shifts(n_angles, n_dist, rng, amplitude=2.0):
    """Sub-pixel sample shifts t_kj ~ U(-amplitude, amplitude) px per axis: [K][J][2] (y, x)."""
    return rng.uniform(-amplitude, amplitude, size=(n_angles, n_dist, 2))


def poisson_amplitude(intensity, mean_counts, rng):
    """sqrt of Poisson-noisy intensity: d_noisy = Poisson(c d) / c, c = counts / mean(d).

    mean_counts = 0 returns sqrt(intensity) unchanged (noiseless data)."""
    intensity = np.asarray(intensity, dtype=np.float64)
    if mean_counts <= 0:
        return np.sqrt(intensity)
    c = mean_counts / max(float(intensity.mean()), 1e-300)
    return np.sqrt(rng.poisson(c * intensity) / c)


def perturbed_probe(q, rng, level=0.1):
    """Start-point probe q * (1 + level * complex standard normal)."""
    noise = (rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)) / np.sqrt(2.0)
    return q * (1.0 + level * noise)
