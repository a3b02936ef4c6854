"""Plain FP64 definition of the holography forward model, F2 and its gradients.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Parity pins live in
``tests/test_oracle_pins.py``; every function below is pinned there by something other
than itself (brute-force DFT, closed forms, Theorem t3, dense-matrix adjoints, finite
differences).

Discretisation readings (the paper states the continuous operators only):

R1  D_z(x) = IDFT2( exp(-i pi lambda z (fx^2 + fy^2)) * DFT2(x) ) on the P x P grid,
    f = k/(P dx) with k in [-P/2, P/2), unnormalised forward DFT with e^{-2 pi i},
    inverse with 1/P^2.  This is the transfer function of the Fresnel kernel
    P_z(x) = e^{ikz}/(i lambda z) exp(i pi |x|^2/(lambda z)) (Appendix A, Eq. defPz)
    with the unimodular constant e^{ikz} dropped.
R2  psi is n x n with pixel centres at i - n/2; the P x P grid has centres at
    i - P/2; the detector is the central n x n crop C.  C* is zero embedding.
R3  q lives on the P x P grid and is never interpolated (Sec. 2: interpolating the
    probe is unstable).
R4  (R psi)(x) = ext + sum_taps bilinear weight * (psi - ext) at psi-coordinate
    m~ x - t, taps outside psi's n x n domain dropped.  This is M_{1/m~}(S_t psi):
    M_m f(x) = f(x/m) (Sec. 2, after Eq. fwd_model_cone) and S_t moves content by +t.
    ext = 1 is free space (transmittance 1); ext = 0 is a test mode in which R is
    linear.  The gradient uses the exact transpose R0^T of the linear part.
R5  Probe shifts s_kj (the S_{s_kj}(q) inside D_{omega_j} of Eq. min2 / Eq. min1) are zero
    unless given.  When given, the model is evaluated in the form the paper points to
    after Eq. min2: shifts commute with the other operators, so the shift can leave the
    probe and act on psi and the detector field instead,
        D_zhat( D_omega(S_s q) * M_{1/m~} S_t psi ) = S_s D_zhat( p * M_{1/m~} S_{t - m~ s} psi ),
    with S_s the band-limited (Fourier phase ramp) shift of the P x P grid, so the probe
    is never interpolated (Sec. 2).  For integer s this is exactly the literal expression
    with q rolled by s; for fractional s the two differ only in how the bilinear object
    field is shifted.
R6  r = u - a u/|u| with u/|u| := 0 where |u| = 0.
R8  z_j are the focus-to-sample distances; m~_j = z_j/z_0, omega_j = (z_j-z_0)/m~_j,
    zeta_j = z_j (Z - z_j)/Z (Sec. 2 after Eq. fwd_model_cone3; Theorem t3).
"""

from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft  # library FFT primitive (multi-threaded), as one step of D_z

# Threads of the library FFT (-1: every host core).  Only the timing of the oracle depends
# on it (a single-core timing run sets 1); the arithmetic does not.
FFT_WORKERS = -1


@dataclass(frozen=True)
class Geometry:
    """Instrument geometry and discretisation (Table 1 lists the paper's instrument).

    wavelength, pixel (object-plane pixel size, i.e. detector pixel / m0), Z
    (focus-to-detector) and z (focus-to-sample distances, increasing) in metres.
    n is the psi/detector side, P the padded FFT side.  ext is the free-space value
    of the resample (R4); w_ref weights the reference-image term of Eq. min1.
    """

    wavelength: float
    pixel: float
    Z: float
    z: tuple
    n: int
    P: int
    ext: float = 1.0
    w_ref: float = 1.0

    @property
    def n_dist(self):
        return len(self.z)


def derived_geometry(z, Z):
    """Magnifications and effective distances of the working formula.

    Sec. 2, after Eq. fwd_model_cone3 and Theorem t3 (Appendix A):
    m~_j = z_j / z_0, omega_j = (z_j - z_0) / m~_j, zeta_j = z_j (Z - z_j) / Z,
    m0 = Z / z_0.  The detector-side distance of plane j is zhat_j = zeta_j / m~_j^2.
    """
    z = np.asarray(z, dtype=np.float64)
    z0 = z[0]
    mt = z / z0
    omega = (z - z0) / mt
    zeta = z * (Z - z) / Z
    zhat = zeta / mt**2
    return {"mt": mt, "omega": omega, "zeta": zeta, "zhat": zhat, "m0": Z / z0,
            "m": Z / z}


def spatial_freq(P, dx):
    """Frequencies k/(P dx), k = 0..P/2-1, -P/2..-1 (reading R1)."""
    k = np.arange(P, dtype=np.float64)
    k[k >= P // 2] -= P
    return k / (P * dx)


def propagate(x, z, wavelength, dx):
    """D_z: Fresnel propagation by distance z of a P x P field (Appendix A, Eq. defGz).

    Convolution with the Fresnel kernel, evaluated through its transfer function
    exp(-i pi lambda z |f|^2) (reading R1).
    """
    x = np.asarray(x, dtype=np.complex128)
    P = x.shape[-1]
    assert x.shape[-2] == P
    f = spatial_freq(P, dx)
    H = np.exp(-1j * np.pi * wavelength * z * (f[:, None] ** 2 + f[None, :] ** 2))
    return sfft.ifft2(sfft.fft2(x, workers=FFT_WORKERS) * H, workers=FFT_WORKERS)


def crop(x, n):
    """Detector crop C: the central n x n window of a P x P field (reading R2)."""
    P = x.shape[-1]
    o = P // 2 - n // 2
    return x[..., o:o + n, o:o + n]


def embed(y, P):
    """C*: zero embedding of an n x n field in the centre of a P x P grid (reading R2)."""
    n = y.shape[-1]
    o = P // 2 - n // 2
    out = np.zeros(y.shape[:-2] + (P, P), dtype=np.complex128)
    out[..., o:o + n, o:o + n] = y
    return out


def shift(x, s):
    """S_s: shift of a P x P field by s = (s_y, s_x) pixels, content moving by +s (Eq. min2
    operator S_s; reading R5).  Evaluated as the phase ramp exp(-2 pi i (k_y s_y + k_x s_x)/P)
    on the DFT with k in [-P/2, P/2): a periodic index shift for integer s, band-limited
    interpolation otherwise.  S_s is unitary, S_s* = S_{-s}, and it commutes with D_z."""
    x = np.asarray(x, dtype=np.complex128)
    P = x.shape[-1]
    k = np.arange(P, dtype=np.float64)
    k[k >= P // 2] -= P
    ramp_y = np.exp(-2j * np.pi * k * s[0] / P)
    ramp_x = np.exp(-2j * np.pi * k * s[1] / P)
    return sfft.ifft2(sfft.fft2(x, workers=FFT_WORKERS) * np.outer(ramp_y, ramp_x), workers=FFT_WORKERS)


def moved_object_shift(t, mt, s):
    """The object shift that carries the probe shift s of plane j (reading R5):
    S_{-s} M_{1/m~} S_t psi = M_{1/m~} S_{t - m~ s} psi, since (M_{1/m~} S_t psi)(x) =
    psi(m~ x - t)."""
    return (t[0] - mt * s[0], t[1] - mt * s[1])


def _bilinear_axis(mt, t, n, P):
    """Per-axis bilinear taps of the resample (reading R4).

    For P-grid index X (coordinate X - P/2) the psi index is xi = m~ (X - P/2) - t + n/2;
    the taps are floor(xi) with weight 1 - frac(xi) and floor(xi)+1 with weight frac(xi).
    """
    X = np.arange(P, dtype=np.float64) - P // 2
    xi = mt * X - t + n // 2
    i0 = np.floor(xi).astype(np.int64)
    f = xi - i0
    return ((i0, 1.0 - f), (i0 + 1, f))


def resample(psi, mt, t, P, ext):
    """R psi = M_{1/m~}(S_t psi) on the P x P grid (Eq. min1 operators; reading R4).

    t = (t_y, t_x) in psi pixels.  Returns ext + sum_taps w_y w_x (psi[tap] - ext),
    taps outside the n x n domain dropped.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    n = psi.shape[-1]
    out = np.full((P, P), ext, dtype=np.complex128)
    for iy, wy in _bilinear_axis(mt, t[0], n, P):
        for ix, wx in _bilinear_axis(mt, t[1], n, P):
            my = (iy >= 0) & (iy < n)
            mx = (ix >= 0) & (ix < n)
            vals = np.zeros((P, P), dtype=np.complex128)
            vals[np.ix_(my, mx)] = psi[np.ix_(iy[my], ix[mx])] - ext
            out += np.outer(wy, wx) * vals
    return out


def resample_adjoint(g, mt, t, n):
    """R0^T: exact transpose of the linear part of ``resample`` (weights scattered back).

    The paper writes the adjoint of M_{1/m~} S_t as S_{-t} M*_{1/m~} (Eq. gradpsi and
    the expression for L*); the discrete adjoint of the bilinear map is its transpose.
    """
    g = np.asarray(g, dtype=np.complex128)
    P = g.shape[-1]
    out = np.zeros((n, n), dtype=np.complex128)
    for iy, wy in _bilinear_axis(mt, t[0], n, P):
        for ix, wx in _bilinear_axis(mt, t[1], n, P):
            my = (iy >= 0) & (iy < n)
            mx = (ix >= 0) & (ix < n)
            Y, Xg = np.meshgrid(np.nonzero(my)[0], np.nonzero(mx)[0], indexing="ij")
            w = np.outer(wy[my], wx[mx])
            np.add.at(out, (iy[Y], ix[Xg]), w * g[Y, Xg])
    return out


def probe_at_planes(q, geo):
    """p_j = D_{omega_j}(q): the probe propagated to sample plane j (Eq. fwd_model_cone3)."""
    d = derived_geometry(geo.z, geo.Z)
    return np.stack([propagate(q, d["omega"][j], geo.wavelength, geo.pixel)
                     for j in range(geo.n_dist)])


def reference_field(q, geo):
    """C D_{zeta_0}(q): the probe on the detector without the sample (Sec. 2, the
    reference-image constraint |D_{zeta_0} q|^2 = d~^r)."""
    d = derived_geometry(geo.z, geo.Z)
    return crop(propagate(q, d["zeta"][0], geo.wavelength, geo.pixel), geo.n)


def bin_amplitudes(a, b):
    """Data binning of the hierarchical scheme (Sec. 3, on speeding up): intensities a^2
    averaged over b x b pixel blocks of the last two axes, returned as amplitudes,
    sqrt(mean_{b x b} a^2).  The side must be a multiple of b."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[-1]
    m = n // b
    blocks = (a ** 2).reshape(a.shape[:-2] + (m, b, m, b))
    return np.sqrt(blocks.mean(axis=(-3, -1)))


def _upsample2_axis(x, axis):
    """Linear interpolation to twice as many pixels along `axis` (pixel centres: fine pixel
    2m sits at coarse coordinate m - 1/4, fine pixel 2m + 1 at m + 1/4), edges clamped."""
    x = np.moveaxis(np.asarray(x), axis, -1)
    N = x.shape[-1]
    out = np.empty(x.shape[:-1] + (2 * N,), dtype=np.result_type(x, np.float64))
    for f in range(2 * N):
        c = (f + 0.5) / 2.0 - 0.5
        i0 = int(np.floor(c))
        w = c - i0
        a, b = min(max(i0, 0), N - 1), min(max(i0 + 1, 0), N - 1)
        out[..., f] = (1.0 - w) * x[..., a] + w * x[..., b]
    return np.moveaxis(out, -1, axis)


def upsample2(x):
    """Extrapolation of a recovered field (psi or q) to a grid twice as dense (Sec. 3, on
    speeding up); reading: separable linear interpolation at the fine pixel centres with
    clamped edges."""
    return _upsample2_axis(_upsample2_axis(x, -1), -2)


def initial_probe(sqrt_dref, geo):
    """Initial probe: the reference image propagated back to sample plane 0 (Sec. 2, on the
    initial guess), q0 = D_{-zeta_0}(E sqrt(d~^r)).  Reading: E embeds the n x n amplitude in
    the P x P grid by repeating its edge values (a zero border would add an edge the probe
    does not have); C D_{zeta_0} q0 = sqrt(d~^r) exactly since D_{zeta_0} D_{-zeta_0} = I."""
    n, P = geo.n, geo.P
    lo = P // 2 - n // 2
    a = np.asarray(sqrt_dref, dtype=np.float64)
    ext = np.pad(a, ((lo, P - n - lo), (lo, P - n - lo)), mode="edge").astype(np.complex128)
    d = derived_geometry(geo.z, geo.Z)
    return propagate(ext, -d["zeta"][0], geo.wavelength, geo.pixel)


def _plane_shifts(shifts, probe_shifts, mt, k, j):
    """(object shift, probe shift or None) of plane (k, j) under reading R5."""
    if probe_shifts is None:
        return shifts[k][j], None
    s = probe_shifts[k][j]
    return moved_object_shift(shifts[k][j], mt, s), s


def forward(psi, q, shifts, geo, probe_shifts=None):
    """Detector wavefields
    u_kj = C D_{zeta_j/m~_j^2}( D_{omega_j}(S_{s_kj} q) * M_{1/m~_j} S_{t_kj} psi_k ).

    Eq. fwd_model_cone3 with the shifts of Eq. min1.  psi: [K][n][n] complex, q: [P][P]
    complex, shifts: [K][J][2] (t_y, t_x) pixels; probe_shifts: [K][J][2] (s_y, s_x) or None
    (zero), evaluated as C S_s D_zhat( p_j * M_{1/m~_j} S_{t - m~_j s} psi_k ) (reading R5).
    Returns u: [K][J][n][n] complex128.
    """
    psi = np.asarray(psi, dtype=np.complex128)
    d = derived_geometry(geo.z, geo.Z)
    p = probe_at_planes(q, geo)
    K, J = psi.shape[0], geo.n_dist
    u = np.empty((K, J, geo.n, geo.n), dtype=np.complex128)
    for k in range(K):
        for j in range(J):
            t, s = _plane_shifts(shifts, probe_shifts, d["mt"][j], k, j)
            x = p[j] * resample(psi[k], d["mt"][j], t, geo.P, geo.ext)
            y = propagate(x, d["zhat"][j], geo.wavelength, geo.pixel)
            if s is not None:
                y = shift(y, s)
            u[k, j] = crop(y, geo.n)
    return u


def amplitude_residual(u, a):
    """r = u - a u/|u| (Eq. gradpsi), with u/|u| := 0 where |u| = 0 (reading R6)."""
    u = np.asarray(u, dtype=np.complex128)
    mag = np.abs(u)
    phase = np.divide(u, mag, out=np.zeros_like(u), where=mag > 0)
    return u - a * phase


def intensity_residual(u, d):
    """r1 = 2 (|u|^2 - d) u: the F1 counterpart of r (Eq. min2).  The real gradient of
    (|u|^2 - d)^2 with respect to u is 4 (|u|^2 - d) u = 2 r1, as the real gradient of
    (|u| - a)^2 is 2 r for F2."""
    u = np.asarray(u, dtype=np.complex128)
    return 2.0 * (np.abs(u) ** 2 - d) * u


def _plane_loss_f2(u, a):
    return float(np.sum((np.abs(u) - a) ** 2))


def _plane_loss_f1(u, d):
    return float(np.sum((np.abs(u) ** 2 - d) ** 2))


def functional(psi, q, shifts, sqrt_d, sqrt_dref, geo, probe_shifts=None):
    """F2 of Eq. min1: sum_kj || |u_kj| - sqrt(d~_kj) ||^2 + w_ref || |D_{zeta_0} q| - sqrt(d~^r) ||^2."""
    u = forward(psi, q, shifts, geo, probe_shifts)
    F = float(np.sum((np.abs(u) - sqrt_d) ** 2))
    if geo.w_ref != 0.0:
        uref = reference_field(q, geo)
        F += geo.w_ref * float(np.sum((np.abs(uref) - sqrt_dref) ** 2))
    return F


def functional_f1(psi, q, shifts, d, d_ref, geo, probe_shifts=None):
    """F1 of Eq. min2: sum_kj || |u_kj|^2 - d~_kj ||^2 + w_ref || |D_{zeta_0} q|^2 - d~^r ||^2
    (d are intensities; the paper's reference term has weight 1)."""
    u = forward(psi, q, shifts, geo, probe_shifts)
    F = float(np.sum((np.abs(u) ** 2 - d) ** 2))
    if geo.w_ref != 0.0:
        uref = reference_field(q, geo)
        F += geo.w_ref * float(np.sum((np.abs(uref) ** 2 - d_ref) ** 2))
    return F


def _gradients(psi, q, shifts, data, data_ref, geo, plane_loss, residual, probe_shifts=None):
    """Loss and real gradients for a per-pixel loss of u whose real gradient is 2 residual(u):
    grad_psi_k = 2 sum_j R0_kj^T( conj(p_j) * D_{-zhat_j}(C* r_kj) ),
    grad_q     = 2 [ sum_j D_{-omega_j}( sum_k conj(R_kj psi_k) * D_{-zhat_j}(C* r_kj) )
                     + w_ref D_{-zeta_0}(C* r_ref) ].
    With probe shifts (reading R5), R_kj carries the object shift t - m~_j s_kj and
    D_{-zhat_j} C* r becomes D_{-zhat_j} S_{-s} C* r, the adjoint of C S_s D_{zhat_j}."""
    psi = np.asarray(psi, dtype=np.complex128)
    d = derived_geometry(geo.z, geo.Z)
    lam, dx, n, P = geo.wavelength, geo.pixel, geo.n, geo.P
    p = probe_at_planes(q, geo)
    K, J = psi.shape[0], geo.n_dist
    F = 0.0
    gpsi = np.zeros((K, n, n), dtype=np.complex128)
    G = np.zeros((J, P, P), dtype=np.complex128)
    for k in range(K):
        for j in range(J):
            t, s = _plane_shifts(shifts, probe_shifts, d["mt"][j], k, j)
            Rpsi = resample(psi[k], d["mt"][j], t, P, geo.ext)
            y = propagate(p[j] * Rpsi, d["zhat"][j], lam, dx)
            u = crop(y if s is None else shift(y, s), n)
            F += plane_loss(u, data[k][j])
            r = residual(u, data[k][j])
            e = embed(r, P)
            v = propagate(e if s is None else shift(e, (-s[0], -s[1])), -d["zhat"][j], lam, dx)
            gpsi[k] += 2.0 * resample_adjoint(np.conj(p[j]) * v, d["mt"][j], t, n)
            G[j] += np.conj(Rpsi) * v
    gq = np.zeros((P, P), dtype=np.complex128)
    for j in range(J):
        gq += 2.0 * propagate(G[j], -d["omega"][j], lam, dx)
    if geo.w_ref != 0.0:
        uref = reference_field(q, geo)
        F += geo.w_ref * plane_loss(uref, data_ref)
        rref = residual(uref, data_ref)
        gq += 2.0 * geo.w_ref * propagate(embed(rref, P), -d["zeta"][0], lam, dx)
    return F, gpsi, gq


def gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo, probe_shifts=None):
    """F2 and its gradients (Eq. gradpsi and the probe gradient after it).

    grad_psi_k = 2 sum_j R0_kj^T( conj(p_j) * D_{-zhat_j}(C* r_kj) )
    grad_q     = 2 [ sum_j D_{-omega_j}( sum_k conj(R_kj psi_k) * D_{-zhat_j}(C* r_kj) )
                     + w_ref D_{-zeta_0}(C* r_ref) ]
    with r = u - sqrt(d~) u/|u|.  These are real gradients for <a,b> = Re sum conj(a) b:
    dF(x; h) = Re <grad, h>.
    Probe shifts (reading R5) are optional, as in ``forward``.
    Returns (F, grad_psi [K][n][n], grad_q [P][P]).
    """
    return _gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo, _plane_loss_f2, amplitude_residual,
                      probe_shifts)


def gradients_f1(psi, q, shifts, d, d_ref, geo, probe_shifts=None):
    """F1 (Eq. min2) and its gradients: the chain of ``gradients`` with r replaced by
    r1 = 2 (|u|^2 - d~) u and intensities d~ as data."""
    return _gradients(psi, q, shifts, d, d_ref, geo, _plane_loss_f1, intensity_residual,
                      probe_shifts)


def plane_gradient(psi_k, q, t_kj, sqrt_d_kj, geo, j):
    """One (k, j) plane's loss and contributions to grad_psi_k and to G_j.

    The per-plane terms of ``gradients`` (Eq. gradpsi), used to check sampled planes of
    large workloads one by one.  Returns (loss_kj, dgrad_psi_k [n][n], G_kj [P][P])
    where grad_q = 2 sum_j D_{-omega_j}(sum_k G_kj) + reference term.
    """
    d = derived_geometry(geo.z, geo.Z)
    lam, dx, n, P = geo.wavelength, geo.pixel, geo.n, geo.P
    pj = propagate(q, d["omega"][j], lam, dx)
    Rpsi = resample(psi_k, d["mt"][j], t_kj, P, geo.ext)
    u = crop(propagate(pj * Rpsi, d["zhat"][j], lam, dx), n)
    loss = float(np.sum((np.abs(u) - sqrt_d_kj) ** 2))
    r = amplitude_residual(u, sqrt_d_kj)
    v = propagate(embed(r, P), -d["zhat"][j], lam, dx)
    dgpsi = 2.0 * resample_adjoint(np.conj(pj) * v, d["mt"][j], t_kj, n)
    return loss, dgpsi, np.conj(Rpsi) * v
