"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a brute-force DFT,
closed forms of Fresnel propagation, the identities of Appendix A, the values printed
in Table 1, dense-matrix adjoints built from unit vectors, pure-Python pointwise
loops, and central finite differences.  A dropped term, a wrong sign, a transposed
index or a mis-scaled distance in the oracle fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest

import holo_synth as hs
from oracle import cg, holo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LAM = hs.WORKLOAD_GEOMETRY["wavelength"]
DX = hs.WORKLOAD_GEOMETRY["pixel"]


def _rng(i=0):
    return np.random.Generator(np.random.PCG64(12345 + i))


def _crandn(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _geo(n, P, ext=1.0, w_ref=1.0, z=None):
    g = hs.WORKLOAD_GEOMETRY
    return holo.Geometry(g["wavelength"], g["pixel"], g["Z"], tuple(z or g["z"]), n, P,
                         ext=ext, w_ref=w_ref)


# ---------------------------------------------------------------- geometry (Table 1)

def test_table1_magnifications_match_printed_values():
    """Z / z_j reproduces the magnifications printed in Table 1 to their printed digits."""
    t = json.load(open(os.path.join(GOLDEN, "table1_pxm_geometry.json")))
    z = np.array(t["z_mm"]) * 1e-3
    d = holo.derived_geometry(z, t["Z_m"])
    for m, printed, digits in zip(d["m"], t["printed_magnifications"], t["printed_digits"]):
        assert round(m, digits) == pytest.approx(printed, abs=10 ** -digits * 0.51)
    assert d["m0"] == pytest.approx(300.0, abs=0.06)
    # 15 um detector pixel, 2x2 binning, 10x objective, demagnified by m0: 10 nm (Sec. 3/4)
    pix = t["detector_pixel_um"] * 1e-6 * t["binning_experimental"] / t["objective"] / d["m0"]
    assert pix == pytest.approx(t["pixel_after_magnification_nm"] * 1e-9, rel=1e-3)
    # 17.05 keV photons: lambda = hc / E
    hc = 1.23984198e-6  # eV m
    assert hc / (t["energy_keV"] * 1e3) == pytest.approx(t["wavelength_m"], rel=1e-5)


def test_theorem_t3_distance_identity():
    """zeta_j / m~_j^2 + omega_j = zeta_0 for every j (Theorem t3: psi = 1 must reduce
    to plain cone-beam propagation of the probe).  A wrong power of m~ or a wrong
    omega breaks it."""
    for geom in (hs.WORKLOAD_GEOMETRY, hs.PAPER_GEOMETRY):
        d = holo.derived_geometry(geom["z"], geom["Z"])
        np.testing.assert_allclose(d["zhat"] + d["omega"], d["zeta"][0], rtol=1e-14)
        assert d["omega"][0] == 0.0 and d["mt"][0] == 1.0
    d = holo.derived_geometry(hs.WORKLOAD_GEOMETRY["z"], hs.WORKLOAD_GEOMETRY["Z"])
    np.testing.assert_allclose(1.0 / d["mt"], [1.0, 0.90196, 0.74194, 0.55422], atol=5e-6)


def test_fresnel_sampling_condition_of_workloads():
    """lambda zhat / dx^2 <= P for the smallest workload (transfer-function validity)."""
    d = holo.derived_geometry(hs.WORKLOAD_GEOMETRY["z"], hs.WORKLOAD_GEOMETRY["Z"])
    assert np.all(LAM * d["zhat"] / DX ** 2 <= 256)


# ---------------------------------------------------------------- D_z

def _dft_matrix(P):
    k = np.arange(P)
    return np.exp(-2j * np.pi * np.outer(k, k) / P)


@pytest.mark.parametrize("P", [4, 6, 8, 12])
def test_propagate_equals_bruteforce_dft(P):
    """D_z against a dense-DFT evaluation of the transfer-function definition."""
    rng = _rng(P)
    x = _crandn(rng, P, P)
    z = 3.3e-4
    dx = 2e-8
    W = _dft_matrix(P)
    kk = np.array([k if k < P / 2 else k - P for k in range(P)], dtype=float) / (P * dx)
    H = np.exp(-1j * math.pi * LAM * z * (kk[:, None] ** 2 + kk[None, :] ** 2))
    X = W @ x @ W.T
    ref = np.conj(W) @ (H * X) @ np.conj(W).T / P ** 2
    np.testing.assert_allclose(holo.propagate(x, z, LAM, dx), ref, rtol=0, atol=1e-12)


def test_propagate_gaussian_closed_form():
    """D_z exp(-pi|x|^2/a) = a/(a + i lambda z) exp(-pi|x|^2/(a + i lambda z)).

    Derived from the Fresnel kernel of Appendix A (Eq. defPz).  Pins the chirp sign,
    the lambda z factor and the frequency scaling (a survey-time check gave 4e-16)."""
    P = 256
    z = 4.598248e-4
    a = 400.0 * DX ** 2
    c = (np.arange(P) - P / 2) * DX
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    g = np.exp(-np.pi * r2 / a)
    w = a + 1j * LAM * z
    ref = a / w * np.exp(-np.pi * r2 / w)
    np.testing.assert_allclose(holo.propagate(g, z, LAM, DX), ref, rtol=0, atol=1e-12)
    # the opposite chirp sign is far off
    bad = a / np.conj(w) * np.exp(-np.pi * r2 / np.conj(w))
    assert np.abs(holo.propagate(g, z, LAM, DX) - bad).max() > 1e-2


def test_propagate_unitary_identity_group_adjoint():
    rng = _rng(1)
    P = 64
    x, y = _crandn(rng, P, P), _crandn(rng, P, P)
    a, b = 2.1e-4, -0.7e-4
    Dx = holo.propagate(x, a, LAM, DX)
    assert np.linalg.norm(Dx) == pytest.approx(np.linalg.norm(x), rel=1e-13)   # Parseval
    np.testing.assert_allclose(holo.propagate(x, 0.0, LAM, DX), x, atol=1e-13)  # D_0 = I
    np.testing.assert_allclose(holo.propagate(Dx, b, LAM, DX),
                               holo.propagate(x, a + b, LAM, DX), atol=1e-12)  # group law
    lhs = np.vdot(Dx, y)
    rhs = np.vdot(x, holo.propagate(y, -a, LAM, DX))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)                                   # D* = D_-z


# ---------------------------------------------------------------- resample

def _pointwise_resample(psi, mt, t, P, ext):
    """Pure-Python loop restatement of reading R4 for tiny sizes."""
    n = psi.shape[0]
    out = np.empty((P, P), dtype=complex)
    for Y in range(P):
        for X in range(P):
            sy = mt * (Y - P // 2) - t[0] + n // 2
            sx = mt * (X - P // 2) - t[1] + n // 2
            iy, ix = math.floor(sy), math.floor(sx)
            fy, fx = sy - iy, sx - ix
            acc = ext
            for dy, wy in ((0, 1 - fy), (1, fy)):
                for dxx, wx in ((0, 1 - fx), (1, fx)):
                    yy, xx = iy + dy, ix + dxx
                    if 0 <= yy < n and 0 <= xx < n:
                        acc += wy * wx * (psi[yy, xx] - ext)
            out[Y, X] = acc
    return out


@pytest.mark.parametrize("mt,t,ext", [(1.0, (0.0, 0.0), 1.0), (1.3, (0.4, -1.7), 1.0),
                                      (1.8043, (-1.2, 0.9), 0.0), (1.0, (2.0, -1.0), 0.0)])
def test_resample_pointwise(mt, t, ext):
    rng = _rng(7)
    psi = _crandn(rng, 6, 6)
    np.testing.assert_allclose(holo.resample(psi, mt, t, 12, ext),
                               _pointwise_resample(psi, mt, t, 12, ext), atol=1e-14)


def test_resample_special_cases():
    rng = _rng(2)
    n, P = 16, 32
    psi = _crandn(rng, n, n)
    # free space: psi = 1 gives exactly 1 (weights sum to one)
    np.testing.assert_allclose(holo.resample(np.ones((n, n)), 1.37, (0.3, -1.2), P, 1.0), 1.0,
                               atol=1e-15)
    # m~ = 1, t = 0 is the identity on the detector window
    np.testing.assert_allclose(holo.crop(holo.resample(psi, 1.0, (0, 0), P, 1.0), n), psi,
                               atol=1e-15)
    # integer shift moves content by +t pixels
    out = holo.crop(holo.resample(psi, 1.0, (2.0, -3.0), P, 0.0), n)
    np.testing.assert_allclose(out[2:, :n - 3], psi[:n - 2, 3:], atol=1e-15)


def test_resample_adjoint_dot_product():
    rng = _rng(3)
    n, P = 10, 24
    psi, g = _crandn(rng, n, n), _crandn(rng, P, P)
    for mt, t in [(1.0, (0.25, -0.5)), (1.55, (1.9, -1.1)), (1.0, (0.0, 0.0))]:
        lhs = np.vdot(holo.resample(psi, mt, t, P, 0.0), g)
        rhs = np.vdot(psi, holo.resample_adjoint(g, mt, t, n))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_proposition_p1_on_gaussian():
    """M_m D_zeta g = D_{zeta m^2} M_m g (Proposition p1, exact for a Gaussian with the
    unimodular constant dropped).  The discrete magnification is the bilinear resample
    with m~ = 1/m; agreement is to the bilinear interpolation error, bounded per axis by
    h^2/8 max|f''| with h = 1 px and f'' <= 2 pi |1/w| for exp(-pi x^2/w)."""
    P = 256
    m = 1.0 / 1.35
    zeta = 3.0e-4
    a = 2000.0 * DX ** 2
    c = (np.arange(P) - P / 2) * DX
    r2 = c[:, None] ** 2 + c[None, :] ** 2
    g = np.exp(-np.pi * r2 / a)
    lhs = holo.resample(holo.propagate(g, zeta, LAM, DX), 1.0 / m, (0, 0), P, 0.0)
    rhs = holo.propagate(holo.resample(g, 1.0 / m, (0, 0), P, 0.0), zeta * m ** 2, LAM, DX)
    w = a + 1j * LAM * zeta
    exact = a / w * np.exp(-np.pi * r2 / (m ** 2 * w))
    bound = 2 * (1.0 / 8.0) * 2 * np.pi * DX ** 2 / abs(w) * 1.1
    assert np.abs(lhs - exact).max() < bound
    assert np.abs(rhs - exact).max() < bound
    # magnifying the other way is far off
    wrong = holo.resample(holo.propagate(g, zeta, LAM, DX), m, (0, 0), P, 0.0)
    assert np.abs(wrong - exact).max() > 50 * bound


# ---------------------------------------------------------------- forward model

def _small_problem(n=16, P=32, K=3, ext=1.0, w_ref=1.0, seed=4, noiseless=False):
    rng = _rng(seed)
    geo = _geo(n, P, ext=ext, w_ref=w_ref)
    psi = hs.transmittance(-rng.uniform(0, 1, (K, n, n)))
    q = hs.striped_probe(P, 0.3 * n, rng)
    t = hs.sample_shifts(K, geo.n_dist, rng)
    if noiseless:
        sqrt_d = np.abs(holo.forward(psi, q, t, geo))
        sqrt_dref = np.abs(holo.reference_field(q, geo))
    else:
        sqrt_d = np.abs(holo.forward(psi, q, t, geo)) * rng.uniform(0.8, 1.2, (K, 4, n, n))
        sqrt_dref = np.abs(holo.reference_field(q, geo)) * rng.uniform(0.8, 1.2, (n, n))
    return geo, psi, q, t, sqrt_d, sqrt_dref


def test_theorem_t3_psi_one_gives_reference_image():
    """psi = 1: every plane's modelled field equals C D_{zeta_0} q (Theorem t3; Sec. 2:
    psi = 1 gives the conventional cone-beam form)."""
    geo, _, q, t, _, _ = _small_problem()
    u = holo.forward(np.ones((2, geo.n, geo.n)), q, t[:2], geo)
    ref = holo.reference_field(q, geo)
    for k in range(2):
        for j in range(4):
            np.testing.assert_allclose(u[k, j], ref, atol=1e-12)


def test_q_one_gives_plain_propagation():
    """q = 1: p_j = 1 and u = C D_{zhat_j} R psi (Sec. 2 consistency check)."""
    geo, psi, _, t, _, _ = _small_problem()
    q = np.ones((geo.P, geo.P))
    p = holo.probe_at_planes(q, geo)
    np.testing.assert_allclose(p, 1.0, atol=1e-13)
    d = holo.derived_geometry(geo.z, geo.Z)
    u = holo.forward(psi, q, t, geo)
    for j in range(4):
        x = holo.resample(psi[1], d["mt"][j], t[1][j], geo.P, 1.0)
        np.testing.assert_allclose(u[1, j], holo.crop(holo.propagate(x, d["zhat"][j], LAM, DX),
                                                      geo.n), atol=1e-12)


def test_dense_matrix_adjoint_and_gradient():
    """Brute force at P = 8, n = 4 in ext = 0 mode: build L_kj and Q_kj as dense matrices
    from unit vectors, and check the oracle gradients equal 2 A^H r (Eq. gradpsi)."""
    n, P = 4, 8
    rng = _rng(5)
    geo = _geo(n, P, ext=0.0, w_ref=0.0)
    psi = _crandn(rng, 1, n, n)
    q = _crandn(rng, P, P)
    t = rng.uniform(-1, 1, (1, 4, 2))
    a = rng.uniform(0.1, 1.0, (1, 4, n, n))
    F, gpsi, gq = holo.gradients(psi, q, t, a, None, geo)
    u = holo.forward(psi, q, t, geo)
    r = holo.amplitude_residual(u, a)
    gpsi_ref = np.zeros(n * n, complex)
    gq_ref = np.zeros(P * P, complex)
    for j in range(4):
        geo_j = _geo(n, P, ext=0.0, w_ref=0.0, z=None)
        Lp = np.zeros((n * n, n * n), complex)
        for c in range(n * n):
            e = np.zeros(n * n, complex)
            e[c] = 1.0
            Lp[:, c] = holo.forward(e.reshape(1, n, n), q, t, geo_j)[0, j].ravel()
        Lq = np.zeros((n * n, P * P), complex)
        for c in range(P * P):
            e = np.zeros(P * P, complex)
            e[c] = 1.0
            Lq[:, c] = holo.forward(psi, e.reshape(P, P), t, geo_j)[0, j].ravel()
        np.testing.assert_allclose(Lp @ psi[0].ravel(), u[0, j].ravel(), atol=1e-12)
        np.testing.assert_allclose(Lq @ q.ravel(), u[0, j].ravel(), atol=1e-12)
        gpsi_ref += 2 * Lp.conj().T @ r[0, j].ravel()
        gq_ref += 2 * Lq.conj().T @ r[0, j].ravel()
    assert F == pytest.approx(np.sum((np.abs(u) - a) ** 2), rel=1e-13)
    np.testing.assert_allclose(gpsi[0].ravel(), gpsi_ref, atol=1e-11)
    np.testing.assert_allclose(gq.ravel(), gq_ref, atol=1e-11)


def test_residual_convention_at_zero_field():
    u = np.array([0.0 + 0j, 3.0 + 4j])
    np.testing.assert_allclose(holo.amplitude_residual(u, np.array([2.0, 2.0])),
                               [0.0, (3 + 4j) * (1 - 2 / 5)], atol=1e-15)


# ---------------------------------------------------------------- functional, gradients

def test_loss_zero_and_gradient_zero_at_truth():
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(noiseless=True)
    F, gpsi, gq = holo.gradients(psi, q, t, sqrt_d, sqrt_dref, geo)
    assert F < 1e-24
    _, gpsi1, gq1 = holo.gradients(np.ones_like(psi), q, t, sqrt_d, sqrt_dref, geo)
    assert np.linalg.norm(gpsi) <= 1e-12 * np.linalg.norm(gpsi1)
    assert np.linalg.norm(gq) <= 1e-12 * np.linalg.norm(gq1)


def test_scale_invariance_and_gradient_identities_ext0():
    """ext = 0, w_ref = 0: L is bilinear in (psi, q) so F(c psi, q / c) = F(psi, q), and its
    derivative in c gives Re<grad_psi, psi> = Re<grad_q, q> and the same with i psi, i q."""
    geo, psi, q, t, sqrt_d, _ = _small_problem(ext=0.0, w_ref=0.0)
    F0 = holo.functional(psi, q, t, sqrt_d, None, geo)
    c = 0.7 - 0.4j
    assert holo.functional(c * psi, q / c, t, sqrt_d, None, geo) == pytest.approx(F0, rel=1e-12)
    _, gpsi, gq = holo.gradients(psi, q, t, sqrt_d, None, geo)
    a1, b1 = cg.re_inner(gpsi, psi), cg.re_inner(gq, q)
    a2, b2 = cg.re_inner(gpsi, 1j * psi), cg.re_inner(gq, 1j * q)
    assert a1 == pytest.approx(b1, rel=1e-10)
    assert a2 == pytest.approx(b2, rel=1e-9, abs=1e-12 * abs(a1))


@pytest.mark.parametrize("ext,w_ref", [(1.0, 1.0), (0.0, 0.0), (1.0, 0.0)])
def test_gradients_central_finite_differences(ext, w_ref):
    """(F(x + e h) - F(x - e h)) / 2e = Re<grad, h> for random directions h."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(ext=ext, w_ref=w_ref)
    F, gpsi, gq = holo.gradients(psi, q, t, sqrt_d, sqrt_dref, geo)
    rng = _rng(9)
    for _ in range(6):
        hpsi, hq = _crandn(rng, *psi.shape), _crandn(rng, *q.shape)
        eps = 1e-6
        fp = holo.functional(psi + eps * hpsi, q + eps * hq, t, sqrt_d, sqrt_dref, geo)
        fm = holo.functional(psi - eps * hpsi, q - eps * hq, t, sqrt_d, sqrt_dref, geo)
        fd = (fp - fm) / (2 * eps)
        an = cg.re_inner(gpsi, hpsi) + cg.re_inner(gq, hq)
        assert fd == pytest.approx(an, rel=1e-7)


@pytest.mark.parametrize("ext,w_ref", [(1.0, 1.0), (0.0, 0.0), (1.0, 0.0)])
def test_f1_gradients_central_finite_differences(ext, w_ref):
    """F1 (Eq. min2, intensities as data): central differences of the functional equal
    Re<grad, h>, which pins r1 = 2 (|u|^2 - d) u through the shared adjoint chain."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(ext=ext, w_ref=w_ref)
    d, dref = sqrt_d ** 2, (sqrt_dref ** 2 if sqrt_dref is not None else None)
    F, gpsi, gq = holo.gradients_f1(psi, q, t, d, dref, geo)
    assert F == pytest.approx(holo.functional_f1(psi, q, t, d, dref, geo), rel=1e-13)
    rng = _rng(19)
    for _ in range(6):
        hpsi, hq = _crandn(rng, *psi.shape), _crandn(rng, *q.shape)
        eps = 1e-6
        fp = holo.functional_f1(psi + eps * hpsi, q + eps * hq, t, d, dref, geo)
        fm = holo.functional_f1(psi - eps * hpsi, q - eps * hq, t, d, dref, geo)
        fd = (fp - fm) / (2 * eps)
        an = cg.re_inner(gpsi, hpsi) + cg.re_inner(gq, hq)
        assert fd == pytest.approx(an, rel=1e-7)


def test_f1_pixel_gradient_closed_form():
    """For one pixel, (|u|^2 - d)^2 has real gradient 4 (|u|^2 - d) u = 2 r1: checked against
    the derivative along 1 and i written out by hand."""
    rng = _rng(23)
    for _ in range(20):
        u = complex(rng.standard_normal(), rng.standard_normal())
        dd = rng.uniform(0.0, 2.0)
        r1 = complex(holo.intensity_residual(np.array([u]), dd)[0])
        f = lambda z: (abs(z) ** 2 - dd) ** 2
        # d f(u + s)/ds at s = 0 for real s is 2 (|u|^2 - d) * 2 Re(u); for imaginary s it is
        # 2 (|u|^2 - d) * 2 Im(u); the real gradient g has Re<g, 1> and Re<g, i> equal to those
        g = 2 * r1
        assert (g.conjugate() * 1).real == pytest.approx(4 * (abs(u) ** 2 - dd) * u.real, rel=1e-12)
        assert (g.conjugate() * 1j).real == pytest.approx(4 * (abs(u) ** 2 - dd) * u.imag, rel=1e-12)
        h = 1e-6
        assert (f(u + h) - f(u - h)) / (2 * h) == pytest.approx((g.conjugate()).real, rel=1e-6)


def test_f1_loss_zero_and_gradient_zero_at_truth():
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(noiseless=True)
    d, dref = sqrt_d ** 2, sqrt_dref ** 2
    F, gpsi, gq = holo.gradients_f1(psi, q, t, d, dref, geo)
    assert F < 1e-24
    _, gpsi1, gq1 = holo.gradients_f1(np.ones_like(psi), q, t, d, dref, geo)
    assert np.linalg.norm(gpsi) <= 1e-12 * np.linalg.norm(gpsi1)
    assert np.linalg.norm(gq) <= 1e-12 * np.linalg.norm(gq1)


def test_plane_gradient_decomposition():
    """Per-plane terms summed over (k, j) reproduce the full gradient."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(w_ref=0.0)
    F, gpsi, gq = holo.gradients(psi, q, t, sqrt_d, None, geo)
    d = holo.derived_geometry(geo.z, geo.Z)
    Ft, gp, G = 0.0, np.zeros_like(gpsi), np.zeros((4, geo.P, geo.P), complex)
    for k in range(psi.shape[0]):
        for j in range(4):
            l, dg, Gk = holo.plane_gradient(psi[k], q, t[k][j], sqrt_d[k][j], geo, j)
            Ft += l
            gp[k] += dg
            G[j] += Gk
    gqt = sum(2 * holo.propagate(G[j], -d["omega"][j], LAM, DX) for j in range(4))
    assert Ft == pytest.approx(F, rel=1e-13)
    np.testing.assert_allclose(gp, gpsi, atol=1e-12)
    np.testing.assert_allclose(gqt, gq, atol=1e-12)


# ---------------------------------------------------------------- CG driver

def test_dai_yuan_reproduces_linear_cg_on_quadratic():
    """With an exact line search on f = 1/2 x^T A x - b^T x, DY-CG is linear CG."""
    rng = _rng(11)
    m = 12
    B = rng.standard_normal((m, m))
    A = B @ B.T + m * np.eye(m)
    b = rng.standard_normal(m)
    # textbook linear CG
    x_lin = np.zeros(m)
    r = b - A @ x_lin
    p = r.copy()
    lin = []
    for _ in range(6):
        al = (r @ r) / (p @ A @ p)
        x_lin = x_lin + al * p
        r_new = r - al * (A @ p)
        p = r_new + (r_new @ r_new) / (r @ r) * p
        r = r_new
        lin.append(x_lin.copy())
    # DY with exact step on the quadratic
    x = np.zeros(m)
    g = A @ x - b
    eta = -g
    for it in range(6):
        gam = -(g @ eta) / (eta @ A @ eta)
        x = x + gam * eta
        g_new = A @ x - b
        eta, _ = cg.dai_yuan_direction(g_new, g, eta)
        g = g_new
        np.testing.assert_allclose(x, lin[it], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("rule", ["fletcher-reeves", "polak-ribiere", "dai-yuan"])
def test_cg_rules_reproduce_linear_cg_on_quadratic(rule):
    """With an exact line search on f = 1/2 x^T A x - b^T x the Fletcher-Reeves,
    Polak-Ribiere-Polyak and Dai-Yuan formulas all give the iterates of textbook linear CG."""
    rng = _rng(12)
    m = 10
    B = rng.standard_normal((m, m))
    A = B @ B.T + m * np.eye(m)
    b = rng.standard_normal(m)
    x_lin, r = np.zeros(m), b.copy()
    p = r.copy()
    lin = []
    for _ in range(5):
        al = (r @ r) / (p @ A @ p)
        x_lin = x_lin + al * p
        r_new = r - al * (A @ p)
        p = r_new + (r_new @ r_new) / (r @ r) * p
        r = r_new
        lin.append(x_lin.copy())
    x = np.zeros(m)
    g = A @ x - b
    eta = -g
    for it in range(5):
        gam = -(g @ eta) / (eta @ A @ eta)
        x = x + gam * eta
        g_new = A @ x - b
        eta, beta = cg.direction(g_new, g, eta, rule)
        assert beta > 0
        g = g_new
        np.testing.assert_allclose(x, lin[it], rtol=1e-10, atol=1e-12)


def test_prp_restarts_when_the_gradient_repeats():
    """Polak-Ribiere-Polyak vanishes when the gradient does not change (its automatic restart);
    Fletcher-Reeves is then 1; for g_new = 0 both vanish."""
    rng = _rng(17)
    g = _crandn(rng, 5, 4)
    assert cg.polak_ribiere_beta(g, g) == pytest.approx(0.0, abs=1e-14)
    assert cg.fletcher_reeves_beta(g, g) == pytest.approx(1.0, rel=1e-14)
    assert cg.polak_ribiere_beta(2 * g, g) == pytest.approx(2.0, rel=1e-14)  # (4 - 2) |g|^2 / |g|^2
    assert cg.fletcher_reeves_beta(np.zeros_like(g), g) == 0.0


def test_armijo_accepts_only_sufficient_decrease():
    """On f(x) = |x|^2 with a steepest-descent direction the Armijo rule accepts the first
    halving of gamma0 that meets f(x + g eta) <= f(x) + c g slope, and returns 0 for an ascent
    direction."""
    f = lambda v: float(np.sum(np.abs(v) ** 2))
    x = np.array([3.0 + 1.0j, -2.0])
    grad = 2 * x
    eta = -grad
    slope = cg.re_inner(grad, eta)
    gam, fx = cg.armijo(f, f(x), slope, x, eta, 4.0, 20, c=0.3)
    # f(x - 2 g x) = (1 - 2 g)^2 f(x); sufficient decrease needs (1 - 2g)^2 <= 1 - 1.2 g,
    # i.e. g <= 0.7; halving from 4 gives 0.5
    assert gam == 0.5 and fx == pytest.approx(0.0)
    assert cg.armijo(f, f(x), cg.re_inner(grad, -eta), x, -eta, 1.0, 20) == (0.0, f(x))


@pytest.mark.parametrize("rule,ls", [("dai-yuan", "armijo"), ("fletcher-reeves", "backtracking"),
                                     ("polak-ribiere", "armijo")])
def test_reconstruction_variants_are_monotone(rule, ls):
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(n=16, P=32, K=2, noiseless=True, seed=6)
    rng = _rng(13)
    out = cg.reconstruct(np.ones_like(psi), hs.perturbed_probe(q, rng), t, sqrt_d, sqrt_dref,
                         geo, iters=4, rule=rule, line_search=ls)
    F = np.array(out["hist"]["F"])
    assert np.all(np.diff(F) <= 0.0) and F[-1] < F[0]


def test_initial_probe_reproduces_reference_amplitude():
    """q0 = D_{-zeta_0}(E sqrt(d~^r)): propagating it forward by zeta_0 returns the edge-padded
    reference amplitude, whose detector crop is sqrt(d~^r) (Sec. 2, initial guess)."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(n=16, P=32, K=1, seed=3)
    q0 = holo.initial_probe(sqrt_dref, geo)
    back = holo.propagate(q0, holo.derived_geometry(geo.z, geo.Z)["zeta"][0], geo.wavelength,
                          geo.pixel)
    np.testing.assert_allclose(holo.crop(back, geo.n), sqrt_dref, atol=1e-12)
    lo = geo.P // 2 - geo.n // 2
    # border rows repeat the first / last data row, border corners the corner value
    np.testing.assert_allclose(back[0, lo:lo + geo.n], sqrt_dref[0], atol=1e-12)
    np.testing.assert_allclose(back[-1, lo:lo + geo.n], sqrt_dref[-1], atol=1e-12)
    assert abs(back[0, 0] - sqrt_dref[0, 0]) < 1e-12 and abs(back[0].imag).max() < 1e-12
    np.testing.assert_allclose(holo.reference_field(q0, geo), sqrt_dref, atol=1e-12)


def test_bin_amplitudes_conserves_intensity_and_constants():
    """Binning averages intensities: a constant stays, block-constant intensities bin exactly,
    and the mean intensity is preserved."""
    rng = _rng(29)
    a = rng.uniform(0.2, 2.0, (3, 16, 16))
    for b in (1, 2, 4, 8):
        ab = holo.bin_amplitudes(a, b)
        assert ab.shape == (3, 16 // b, 16 // b)
        assert np.mean(ab ** 2) == pytest.approx(np.mean(a ** 2), rel=1e-13)
    np.testing.assert_allclose(holo.bin_amplitudes(np.full((8, 8), 1.7), 4), 1.7, rtol=1e-14)
    blocks = rng.uniform(0.5, 1.5, (4, 4))
    fine = np.sqrt(np.kron(blocks ** 2, np.ones((2, 2))))
    np.testing.assert_allclose(holo.bin_amplitudes(fine, 2), np.sqrt(blocks ** 2), rtol=1e-14)


def test_upsample2_is_linear_interpolation_at_pixel_centres():
    """Twice-as-dense extrapolation: constants stay, a linear ramp is reproduced at the
    interior fine pixel centres (coarse coordinate (f + 1/2)/2 - 1/2), the edges are clamped,
    and the mean of each fine pixel pair is the [1/8, 3/4, 1/8] smoothing of the coarse row."""
    N = 9
    ramp = 0.3 * np.arange(N) - 1.1
    up = holo.upsample2(np.tile(ramp, (N, 1)))
    f = np.arange(2 * N)
    want = 0.3 * ((f + 0.5) / 2 - 0.5) - 1.1
    np.testing.assert_allclose(up[4, 1:-1], want[1:-1], rtol=1e-13, atol=1e-14)
    assert up[4, 0] == pytest.approx(ramp[0]) and up[4, -1] == pytest.approx(ramp[-1])
    np.testing.assert_allclose(holo.upsample2(np.full((5, 5), 2.0 - 1.0j)), 2.0 - 1.0j, rtol=1e-14)
    rng = _rng(31)
    x = rng.standard_normal(N)
    u = holo._upsample2_axis(x, -1)
    pair = 0.5 * (u[0::2] + u[1::2])
    np.testing.assert_allclose(pair[1:-1], 0.125 * x[:-2] + 0.75 * x[1:-1] + 0.125 * x[2:], rtol=1e-13)


def test_hierarchical_reconstruction_levels():
    """The hierarchical driver: one level without binning is the plain driver from psi = 1 and
    the initial probe; with binning every level is monotone, sizes double, and the last level
    works on the full grid."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(n=32, P=64, K=2, noiseless=True, seed=8)
    one = cg.reconstruct_hierarchical(sqrt_d, sqrt_dref, t, geo, [(1, 3)])
    ref = cg.reconstruct(np.ones_like(psi), holo.initial_probe(sqrt_dref, geo), t, sqrt_d,
                         sqrt_dref, geo, 3)
    np.testing.assert_allclose(one[0]["hist"]["F"], ref["hist"]["F"], rtol=1e-13)
    lev = cg.reconstruct_hierarchical(sqrt_d, sqrt_dref, t, geo, [(4, 3), (2, 3), (1, 3)])
    assert [r["psi"].shape[-1] for r in lev] == [8, 16, 32] and lev[-1]["q"].shape == (64, 64)
    for r in lev:
        F = np.array(r["hist"]["F"])
        assert np.all(np.diff(F) <= 0.0)


def test_reconstruction_is_monotone():
    """The line search never lets F increase (Sec. 2, after Eq. DaiYuan2)."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(n=16, P=32, K=2, noiseless=True, seed=6)
    rng = _rng(13)
    out = cg.reconstruct(np.ones_like(psi), hs.perturbed_probe(q, rng), t, sqrt_d, sqrt_dref,
                         geo, iters=4)
    F = np.array(out["hist"]["F"])
    assert np.all(np.diff(F) <= 0.0)
    assert F[-1] < F[0]


# ---------------------------------------------------------------- probe shifts (reading R5)

def test_shift_is_index_roll_for_integers_and_moves_a_gaussian():
    """S_s moves content by +s: an integer s is a periodic index roll, and a fractional s
    moves a band-limited Gaussian to its samples at x - s (sign and scale of the ramp)."""
    rng = _rng(21)
    P = 32
    x = _crandn(rng, P, P)
    for s in [(1, 0), (0, -3), (2, 5), (-7, 4)]:
        np.testing.assert_allclose(holo.shift(x, s), np.roll(x, s, axis=(0, 1)), atol=1e-13)
    P, sig = 64, 3.0
    c = np.arange(P) - P // 2
    g = lambda y0, x0: np.exp(-((c[:, None] - y0) ** 2 + (c[None, :] - x0) ** 2) / (2 * sig**2))
    s = (0.37, -1.61)
    np.testing.assert_allclose(holo.shift(g(0, 0), s), g(*s), atol=1e-12)
    assert np.abs(holo.shift(g(0, 0), (-s[0], -s[1])) - g(*s)).max() > 0.1


def test_shift_group_unitary_adjoint_and_commutes_with_propagation():
    rng = _rng(22)
    P = 32
    x, y = _crandn(rng, P, P), _crandn(rng, P, P)
    a, b = (0.3, -1.2), (1.45, 0.7)
    np.testing.assert_allclose(holo.shift(holo.shift(x, a), b),
                               holo.shift(x, (a[0] + b[0], a[1] + b[1])), atol=1e-12)
    assert np.linalg.norm(holo.shift(x, a)) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    lhs = np.vdot(holo.shift(x, a), y)
    rhs = np.vdot(x, holo.shift(y, (-a[0], -a[1])))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    z = 4.6e-4
    np.testing.assert_allclose(holo.shift(holo.propagate(x, z, LAM, DX), a),
                               holo.propagate(holo.shift(x, a), z, LAM, DX), atol=1e-12)


def _literal_forward_rolled_probe(psi, q, t, s, geo):
    """Eq. min1's field with the probe shift applied literally, S_s q = np.roll(q, s) for
    integer s, written without the moved form."""
    d = holo.derived_geometry(geo.z, geo.Z)
    K, J = psi.shape[0], geo.n_dist
    u = np.empty((K, J, geo.n, geo.n), complex)
    for k in range(K):
        for j in range(J):
            qs = np.roll(q, (int(s[k][j][0]), int(s[k][j][1])), axis=(0, 1))
            pj = holo.propagate(qs, d["omega"][j], LAM, DX)
            x = pj * holo.resample(psi[k], d["mt"][j], t[k][j], geo.P, geo.ext)
            u[k, j] = holo.crop(holo.propagate(x, d["zhat"][j], LAM, DX), geo.n)
    return u


@pytest.mark.parametrize("ext", [1.0, 0.0])
def test_probe_shift_integer_equals_rolled_probe(ext):
    """The moved form (reading R5) is the literal D_omega(S_s q) of Eq. min1 exactly when s
    is an integer shift: S_s q is then q rolled by s."""
    geo, psi, q, t, _, _ = _small_problem(ext=ext)
    rng = _rng(23)
    s = rng.integers(-3, 4, (psi.shape[0], geo.n_dist, 2)).astype(float)
    u = holo.forward(psi, q, t, geo, probe_shifts=s)
    np.testing.assert_allclose(u, _literal_forward_rolled_probe(psi, q, t, s, geo), atol=1e-12)
    # the object shift must carry -m~ s: without it the fields differ at O(1)
    d = holo.derived_geometry(geo.z, geo.Z)
    assert np.abs(u - holo.forward(psi, q, t, geo)).max() > 1e-2
    assert d["mt"][3] > 1.5


def test_probe_shift_zero_and_psi_one():
    """Zero probe shifts give the unshifted model; psi = 1 gives C S_s D_{zeta_0} q on every
    plane (Theorem t3 with the shift commuted out of the propagations)."""
    geo, psi, q, t, _, _ = _small_problem()
    K, J = psi.shape[0], geo.n_dist
    zero = np.zeros((K, J, 2))
    np.testing.assert_allclose(holo.forward(psi, q, t, geo, probe_shifts=zero),
                               holo.forward(psi, q, t, geo), atol=1e-13)
    s = _rng(24).integers(-2, 3, (K, J, 2)).astype(float)
    u = holo.forward(np.ones_like(psi), q, t, geo, probe_shifts=s)
    d = holo.derived_geometry(geo.z, geo.Z)
    b = holo.propagate(q, d["zeta"][0], LAM, DX)
    for k in range(K):
        for j in range(J):
            ref = holo.crop(np.roll(b, (int(s[k, j, 0]), int(s[k, j, 1])), axis=(0, 1)), geo.n)
            np.testing.assert_allclose(u[k, j], ref, atol=1e-12)


def test_probe_shift_fractional_close_to_band_limited_probe_shift():
    """For fractional s the moved form differs from D_omega(S_s q) * R_t psi only in how the
    bilinear object field is shifted: on a smooth object the two fields agree to a small
    fraction of the object's contribution, and far worse with the object shift's sign
    flipped."""
    n, P = 32, 64
    geo = _geo(n, P)
    d = holo.derived_geometry(geo.z, geo.Z)
    c = np.arange(n) - n // 2
    phase = -0.8 * np.exp(-(c[:, None] ** 2 + c[None, :] ** 2) / (2 * 5.0 ** 2))
    psi = hs.transmittance(phase)[None]
    q = hs.striped_probe(P, 0.3 * n, _rng(25))
    t = np.array([[[0.6, -1.1]] * 4])
    s = np.array([[[0.45, -0.3], [1.3, 0.2], [-0.7, 0.55], [0.25, 1.6]]])
    u = holo.forward(psi, q, t, geo, probe_shifts=s)
    obj = np.abs(u - holo.forward(np.ones_like(psi), q, t, geo, probe_shifts=s))
    lit = np.empty_like(u)
    wrong = np.empty_like(u)
    for j in range(4):
        pj = holo.propagate(holo.shift(q, s[0, j]), d["omega"][j], LAM, DX)
        x = pj * holo.resample(psi[0], d["mt"][j], t[0, j], P, 1.0)
        lit[0, j] = holo.crop(holo.propagate(x, d["zhat"][j], LAM, DX), n)
        tw = (t[0, j, 0] + d["mt"][j] * s[0, j, 0], t[0, j, 1] + d["mt"][j] * s[0, j, 1])
        y = holo.propagate(holo.probe_at_planes(q, geo)[j] *
                           holo.resample(psi[0], d["mt"][j], tw, P, 1.0), d["zhat"][j], LAM, DX)
        wrong[0, j] = holo.crop(holo.shift(y, s[0, j]), n)
    err = np.linalg.norm(u - lit) / np.linalg.norm(obj)
    assert err < 0.01
    assert np.linalg.norm(wrong - lit) / np.linalg.norm(obj) > 10 * err


@pytest.mark.parametrize("ext,w_ref,f1", [(1.0, 1.0, False), (0.0, 0.0, False), (1.0, 1.0, True)])
def test_probe_shift_gradients_central_finite_differences(ext, w_ref, f1):
    """With fractional probe shifts, central differences of F2 (and F1) equal Re<grad, h>:
    pins the adjoint D_{-zhat} S_{-s} C* and the moved object shift in both gradients."""
    geo, psi, q, t, sqrt_d, sqrt_dref = _small_problem(ext=ext, w_ref=w_ref)
    s = _rng(26).uniform(-2, 2, (psi.shape[0], geo.n_dist, 2))
    fun, grad = ((holo.functional_f1, holo.gradients_f1) if f1 else
                 (holo.functional, holo.gradients))
    data, dref = (sqrt_d ** 2, sqrt_dref ** 2) if f1 else (sqrt_d, sqrt_dref)
    F, gpsi, gq = grad(psi, q, t, data, dref, geo, probe_shifts=s)
    assert F == pytest.approx(fun(psi, q, t, data, dref, geo, probe_shifts=s), rel=1e-13)
    rng = _rng(27)
    for _ in range(4):
        hpsi, hq = _crandn(rng, *psi.shape), _crandn(rng, *q.shape)
        eps = 1e-6
        fp = fun(psi + eps * hpsi, q + eps * hq, t, data, dref, geo, probe_shifts=s)
        fm = fun(psi - eps * hpsi, q - eps * hq, t, data, dref, geo, probe_shifts=s)
        an = cg.re_inner(gpsi, hpsi) + cg.re_inner(gq, hq)
        assert (fp - fm) / (2 * eps) == pytest.approx(an, rel=1e-7)


def test_drivers_with_probe_shifts():
    """The joint driver and the hierarchy carry probe shifts: zero shifts reproduce the
    unshifted F history, F decreases monotonically with fractional shifts, and one level
    without binning is the plain driver from psi = 1 and the initial probe."""
    geo, psi, q, t, _, _ = _small_problem(n=32, P=64, K=2, noiseless=True, seed=8)
    s = _rng(31).uniform(-2, 2, (2, geo.n_dist, 2))
    sqrt_d = np.abs(holo.forward(psi, q, t, geo, probe_shifts=s))
    sqrt_dref = np.abs(holo.reference_field(q, geo))
    q0 = holo.initial_probe(sqrt_dref, geo)
    plain = cg.reconstruct(np.ones_like(psi), q0, t, sqrt_d, sqrt_dref, geo, 3)
    zero = cg.reconstruct(np.ones_like(psi), q0, t, sqrt_d, sqrt_dref, geo, 3,
                          probe_shifts=np.zeros_like(s))
    np.testing.assert_allclose(zero["hist"]["F"], plain["hist"]["F"], rtol=1e-12)
    shifted = cg.reconstruct(np.ones_like(psi), q0, t, sqrt_d, sqrt_dref, geo, 4, probe_shifts=s)
    F = np.array(shifted["hist"]["F"])
    assert np.all(np.diff(F) <= 0.0) and F[-1] < F[0]
    one = cg.reconstruct_hierarchical(sqrt_d, sqrt_dref, t, geo, [(1, 4)], probe_shifts=s)
    np.testing.assert_allclose(one[0]["hist"]["F"], F, rtol=1e-13)
    lev = cg.reconstruct_hierarchical(sqrt_d, sqrt_dref, t, geo, [(2, 2), (1, 2)], probe_shifts=s)
    for r in lev:
        assert np.all(np.diff(r["hist"]["F"]) <= 0.0)


def test_dense_matrix_adjoint_and_gradient_with_probe_shifts():
    """Brute force at P = 8, n = 4 (ext = 0) with fractional probe shifts: the columns of
    L_kj and Q_kj built from unit vectors reproduce the fields, and the oracle gradients equal
    2 A^H r, which pins D_{-zhat} S_{-s} C* as the exact adjoint of C S_s D_{zhat}."""
    n, P = 4, 8
    rng = _rng(41)
    geo = _geo(n, P, ext=0.0, w_ref=0.0)
    psi = _crandn(rng, 1, n, n)
    q = _crandn(rng, P, P)
    t = rng.uniform(-1, 1, (1, 4, 2))
    s = rng.uniform(-1.5, 1.5, (1, 4, 2))
    a = rng.uniform(0.1, 1.0, (1, 4, n, n))
    F, gpsi, gq = holo.gradients(psi, q, t, a, None, geo, probe_shifts=s)
    u = holo.forward(psi, q, t, geo, probe_shifts=s)
    r = holo.amplitude_residual(u, a)
    gpsi_ref = np.zeros(n * n, complex)
    gq_ref = np.zeros(P * P, complex)
    for j in range(4):
        Lp = np.zeros((n * n, n * n), complex)
        for c in range(n * n):
            e = np.zeros(n * n, complex)
            e[c] = 1.0
            Lp[:, c] = holo.forward(e.reshape(1, n, n), q, t, geo, probe_shifts=s)[0, j].ravel()
        Lq = np.zeros((n * n, P * P), complex)
        for c in range(P * P):
            e = np.zeros(P * P, complex)
            e[c] = 1.0
            Lq[:, c] = holo.forward(psi, e.reshape(P, P), t, geo, probe_shifts=s)[0, j].ravel()
        np.testing.assert_allclose(Lp @ psi[0].ravel(), u[0, j].ravel(), atol=1e-12)
        np.testing.assert_allclose(Lq @ q.ravel(), u[0, j].ravel(), atol=1e-12)
        gpsi_ref += 2 * Lp.conj().T @ r[0, j].ravel()
        gq_ref += 2 * Lq.conj().T @ r[0, j].ravel()
    assert F == pytest.approx(np.sum((np.abs(u) - a) ** 2), rel=1e-13)
    np.testing.assert_allclose(gpsi[0].ravel(), gpsi_ref, atol=1e-11)
    np.testing.assert_allclose(gq.ravel(), gq_ref, atol=1e-11)
