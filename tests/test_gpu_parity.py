"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 against the oracle): loss 1e-5, gradients 1e-4, the targets the
FP32-wavefield / FP64-reduction design must meet; fields and single propagations 1e-5.
Inputs come from holo_synth; data are made by the oracle, never by the CUDA path.
"""

import numpy as np
import pytest

import evalpoints as ep
import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY
LOSS_TOL, GRAD_TOL, FIELD_TOL = 1e-5, 1e-4, 1e-5


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def dev(a, dtype):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_problem(n, P, K, J=4, ext=1.0, w_ref=1.0, seed=0, noiseless=False, z=None,
                 point="start"):
    """A seeded problem with oracle-made data.  point: "start" (psi = 1 in production mode
    ext = 1, a random transmittance for ext = 0, and the perturbed probe), "iterated" (after 5
    iterations of the oracle's CG driver from the start point) or "object" (the true object
    times a small perturbation, with the perturbed probe)."""
    rng = hs.rng_for(hs.SEED_BASE + 7, seed)
    z = tuple(z or G["z"][:J])
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], z, n, P, ext=ext, w_ref=w_ref)
    w = hs.Workload("t", n, P, K, J, "ellipses", n * 40.0 / 128, 0.0, K, seed)
    psi_true = hs.object_stack(w, range(K), rng)
    q_true = hs.striped_probe(P, n * 40.0 / 128, rng)
    t = hs.sample_shifts(K, J, rng).astype(np.float32).astype(np.float64)
    sqrt_d = np.abs(oh.forward(psi_true, q_true, t, geo))
    sqrt_dref = np.abs(oh.reference_field(q_true, geo))
    if not noiseless:
        sqrt_d = hs.poisson_amplitude(sqrt_d ** 2, 1e4, rng)
        sqrt_dref = hs.poisson_amplitude(sqrt_dref ** 2, 1e4, rng)
    psi0 = np.ones((K, n, n), np.complex128) if ext == 1.0 else hs.transmittance(
        -0.5 * rng.uniform(0, 1, (K, n, n)))
    q0 = hs.perturbed_probe(q_true, rng)
    # evaluation points are rounded to complex64 so both sides see the same inputs
    psi0 = psi0.astype(np.complex64).astype(np.complex128)
    q0 = q0.astype(np.complex64).astype(np.complex128)
    sqrt_d = sqrt_d.astype(np.float32).astype(np.float64)
    sqrt_dref = sqrt_dref.astype(np.float32).astype(np.float64)
    if point == "iterated":
        psi0, q0 = ep.iterated_point(psi0, q0, t, sqrt_d, sqrt_dref, geo)
    elif point == "object":
        psi0 = ep.object_point(psi_true, rng)
    return dict(geo=geo, psi=psi0, q=q0, t=t, sqrt_d=sqrt_d, sqrt_dref=sqrt_dref,
                psi_true=psi_true, q_true=q_true)


def make_holo(pr, chunk=0):
    from paper_2407_20304_gb300 import Holo
    geo = pr["geo"]
    K = pr["psi"].shape[0]
    h = Holo(geo.n, K, geo.n_dist, geo.wavelength, geo.pixel, geo.Z, geo.z, pad=geo.P,
             chunk=chunk, w_ref=geo.w_ref, ext=geo.ext)
    h.set_shifts(pr["t"].astype(np.float32))
    h.set_data(dev(pr["sqrt_d"], torch.float32),
               dev(pr["sqrt_dref"], torch.float32) if geo.w_ref else None)
    h.set_probe(dev(pr["q"], torch.complex64))
    return h


# ------------------------------------------------------------------ D_z

@pytest.mark.parametrize("P", [16, 32, 64, 128, 256, 512, 1024, 2048, 4096,
                               48, 96, 192, 384, 768, 1536, 3072])
def test_propagate_matches_oracle(P):
    from paper_2407_20304_gb300 import Holo
    n = max(16, P // 2)
    rng = np.random.default_rng(P)
    x = (rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P))).astype(np.complex64)
    h = Holo(n, 1, 1, G["wavelength"], G["pixel"], G["Z"], G["z"][:1], pad=P)
    for z in (4.598e-4, -2.1e-4):
        got = h.propagate(dev(x, torch.complex64), z).cpu().numpy()
        ref = oh.propagate(x.astype(np.complex128), z, G["wavelength"], G["pixel"])
        assert rel(got, ref) < FIELD_TOL, (P, z, rel(got, ref))


# ------------------------------------------------------------------ forward

@pytest.mark.parametrize("n,P,K,ext", [(16, 32, 2, 1.0), (32, 64, 3, 0.0), (64, 128, 2, 1.0),
                                       (100, 256, 2, 1.0), (128, 256, 3, 1.0),
                                       (24, 64, 1, 1.0), (24, 48, 2, 1.0), (48, 96, 2, 0.0),
                                       (96, 192, 2, 1.0), (192, 384, 2, 1.0)])
def test_forward_fields_and_loss(n, P, K, ext):
    pr = make_problem(n, P, K, ext=ext, seed=n + K)
    h = make_holo(pr)
    u = torch.empty((K, 4, n, n), dtype=torch.complex64, device="cuda")
    loss = h.forward(dev(pr["psi"], torch.complex64), u_out=u)
    u_ref = oh.forward(pr["psi"], pr["q"], pr["t"], pr["geo"])
    F_ref = oh.functional(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"], pr["geo"])
    assert rel(u.cpu().numpy(), u_ref) < FIELD_TOL
    assert abs(loss - F_ref) / F_ref < LOSS_TOL


# ------------------------------------------------------------------ gradients

@pytest.mark.parametrize("n,P,K,J,ext,w_ref", [
    (16, 32, 2, 4, 1.0, 1.0), (32, 64, 3, 4, 1.0, 1.0), (32, 64, 2, 4, 0.0, 0.0),
    (64, 128, 2, 4, 1.0, 0.0), (100, 256, 2, 4, 1.0, 1.0), (128, 256, 4, 4, 1.0, 1.0),
    (64, 128, 3, 1, 1.0, 1.0), (48, 128, 2, 3, 1.0, 1.0), (256, 512, 2, 4, 1.0, 1.0),
    # line lengths 3 * 2^k (radix-3 step)
    (24, 48, 2, 4, 1.0, 1.0), (48, 96, 3, 4, 1.0, 1.0), (96, 192, 2, 3, 1.0, 0.0),
    (192, 384, 2, 4, 0.0, 0.0), (384, 768, 2, 4, 1.0, 1.0), (700, 1536, 1, 2, 1.0, 1.0),
    # pass B with TMA-staged Y tiles (whole column-group rounds); n = 1826 leaves the last
    # group of 4 columns half outside the detector
    (1216, 2048, 1, 3, 1.0, 1.0), (1826, 2048, 2, 2, 1.0, 1.0),
])
def test_gradient_matches_oracle(n, P, K, J, ext, w_ref):
    pr = make_problem(n, P, K, J=J, ext=ext, w_ref=w_ref, seed=3 * n + J)
    h = make_holo(pr)
    loss, gp, gq = h.gradient(dev(pr["psi"], torch.complex64))
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"])
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL


# Production mode (ext = 1) away from psi = 1, where the object field w = R0(psi - 1) is not
# zero: every line-length class, the row passes' 3-blocks-per-SM forms (P = 768 .. 4096), the
# plane-split (n <= 1024) and whole-round (n = 1826, 2048) forms of pass B, and the
# group-local last exchange of P = 4096.  Small problems are evaluated after 5 oracle CG
# iterations, large ones at the perturbed true object.
AWAY = [(16, 32, 2, 4, "iterated"), (32, 64, 2, 4, "iterated"), (64, 128, 2, 4, "iterated"),
        (128, 256, 2, 4, "iterated"), (256, 512, 1, 4, "iterated"), (24, 48, 2, 4, "iterated"),
        (48, 96, 2, 4, "iterated"), (96, 192, 2, 3, "iterated"), (192, 384, 1, 4, "iterated"),
        (384, 768, 2, 4, "object"), (512, 1024, 2, 4, "object"), (700, 1536, 1, 2, "object"),
        (1024, 2048, 1, 4, "object"), (1826, 2048, 2, 2, "object"),
        (1536, 3072, 1, 2, "object"), (2048, 4096, 1, 2, "object")]


@pytest.mark.parametrize("n,P,K,J,point", AWAY)
def test_gradient_away_from_start_matches_oracle(n, P, K, J, point):
    pr = make_problem(n, P, K, J=J, seed=11 * n + J, point=point)
    # the object field is far from zero at this point
    assert np.abs(pr["psi"] - 1).mean() > 1e-2
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    loss_f = h.forward(psi)
    loss, gp, gq = h.gradient(psi)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"])
    e = (abs(loss - F) / F, rel(gp.cpu().numpy(), gp_ref), rel(gq.cpu().numpy(), gq_ref))
    print(f"n={n} P={P} {point}: loss {e[0]:.2e}, grad_psi {e[1]:.2e}, grad_q {e[2]:.2e}")
    assert abs(loss_f - F) / F < LOSS_TOL
    assert e[0] < LOSS_TOL and e[1] < GRAD_TOL and e[2] < GRAD_TOL


# Pass B's forms of a partial last round of column groups (holo_set_schedule's pass_b_split):
# 0 whole groups per block, 1 the plane-split kernel, 2 the split inside the staged kernel
# (with the Y stage from P = 1024 up), each against the oracle, forward loss included.
SPLITS = [(64, 128, 2, 4, 0), (64, 128, 2, 4, 2), (100, 256, 2, 4, 1), (384, 768, 2, 4, 2),
          (1024, 2048, 1, 4, 0), (1024, 2048, 1, 4, 1), (1024, 2048, 1, 4, 2),
          (1826, 2048, 2, 2, 2), (1536, 3072, 1, 2, 2), (2048, 4096, 1, 2, 2),
          (2048, 4096, 2, 2, 1)]


@pytest.mark.parametrize("n,P,K,J,split", SPLITS)
def test_pass_b_split_forms_match_oracle(n, P, K, J, split):
    pr = make_problem(n, P, K, J=J, seed=5 * n + J + split, point="object")
    h = make_holo(pr)
    h.set_schedule(0, -1, split)
    psi = dev(pr["psi"], torch.complex64)
    loss_f = h.forward(psi)
    loss, gp, gq = h.gradient(psi)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"])
    e = (abs(loss - F) / F, rel(gp.cpu().numpy(), gp_ref), rel(gq.cpu().numpy(), gq_ref))
    print(f"n={n} P={P} split {split}: loss {e[0]:.2e}, grad_psi {e[1]:.2e}, grad_q {e[2]:.2e}")
    assert abs(loss_f - F) / F < LOSS_TOL
    assert e[0] < LOSS_TOL and e[1] < GRAD_TOL and e[2] < GRAD_TOL
    # a second evaluation reuses the slots: the same results bit for bit
    loss2, gp2, gq2 = h.gradient(psi)
    assert loss2 == loss and torch.equal(gp2, gp) and torch.equal(gq2, gq)
    with pytest.raises(RuntimeError):
        h.set_schedule(0, -1, 3)


@pytest.mark.parametrize("n,P,K,point", [(64, 128, 2, "iterated"), (96, 192, 2, "iterated"),
                                         (1024, 2048, 1, "object")])
def test_forward_fields_away_from_start(n, P, K, point):
    pr = make_problem(n, P, K, seed=13 * n, point=point)
    h = make_holo(pr)
    u = torch.empty((K, 4, n, n), dtype=torch.complex64, device="cuda")
    loss = h.forward(dev(pr["psi"], torch.complex64), u_out=u)
    u_ref = oh.forward(pr["psi"], pr["q"], pr["t"], pr["geo"])
    F_ref = oh.functional(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"], pr["geo"])
    assert rel(u.cpu().numpy(), u_ref) < FIELD_TOL
    assert abs(loss - F_ref) / F_ref < LOSS_TOL


@pytest.mark.parametrize("n,P,K,J,ext,w_ref,point", [
    (16, 32, 2, 4, 1.0, 1.0, "start"), (64, 128, 3, 4, 1.0, 1.0, "start"),
    (48, 96, 2, 3, 0.0, 0.0, "start"),
    (64, 128, 2, 4, 1.0, 1.0, "object"), (384, 768, 1, 4, 1.0, 1.0, "object"),
    (1024, 2048, 1, 2, 1.0, 1.0, "object"),
    (128, 256, 2, 4, 1.0, 1.0, "start"), (256, 512, 2, 2, 1.0, 0.0, "start"),
])
def test_intensity_functional_matches_oracle(n, P, K, J, ext, w_ref, point):
    """F1 (Eq. min2): intensities as data, r = 2 (|u|^2 - d) u; forward loss and gradients
    against the oracle's functional_f1 / gradients_f1."""
    pr = make_problem(n, P, K, J=J, ext=ext, w_ref=w_ref, seed=5 * n + J, point=point)
    d = pr["sqrt_d"] ** 2
    dref = pr["sqrt_dref"] ** 2 if w_ref else None
    h = make_holo(pr)
    h.set_functional("intensity")
    h.set_data(dev(d, torch.float32), dev(dref, torch.float32) if w_ref else None)
    loss_f = h.forward(dev(pr["psi"], torch.complex64))
    loss, gp, gq = h.gradient(dev(pr["psi"], torch.complex64))
    F, gp_ref, gq_ref = oh.gradients_f1(pr["psi"], pr["q"], pr["t"], d, dref, pr["geo"])
    assert abs(loss_f - F) / F < LOSS_TOL and abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL
    h.set_functional("amplitude")
    h.set_data(dev(pr["sqrt_d"], torch.float32), dev(pr["sqrt_dref"], torch.float32) if w_ref else None)
    F2 = oh.functional(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"], pr["geo"])
    assert abs(h.forward(dev(pr["psi"], torch.complex64)) - F2) / F2 < LOSS_TOL


def test_chunks_accumulate_to_full_gradient():
    pr = make_problem(64, 128, 5, seed=11)
    h = make_holo(pr, chunk=2)
    psi = dev(pr["psi"], torch.complex64)
    gp = torch.full_like(psi, float("nan"))     # every slice must be overwritten
    gq = torch.full((128, 128), float("nan"), dtype=torch.complex64, device="cuda")
    loss = 0.0
    for k0 in range(0, 5, 2):
        nk = min(2, 5 - k0)
        loss, _, _ = h.gradient(psi[k0:k0 + nk], grad_psi=gp[k0:k0 + nk], grad_q=gq, k0=k0,
                                accumulate_q=k0 > 0, loss_in=loss)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"])
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL


def test_gradient_host_buffers_match_device_call():
    pr = make_problem(64, 128, 3, seed=5)
    h = make_holo(pr)
    loss_d, gp_d, gq_d = h.gradient(dev(pr["psi"], torch.complex64))
    loss_h, gp_h, gq_h = h.gradient_host(pr["psi"].astype(np.complex64),
                                         sqrt_d=pr["sqrt_d"].astype(np.float32),
                                         q=pr["q"].astype(np.complex64))
    assert loss_h == loss_d
    np.testing.assert_array_equal(gp_h, gp_d.cpu().numpy())
    np.testing.assert_array_equal(gq_h, gq_d.cpu().numpy())


def test_gradient_host_in_parts_matches_device_call():
    """12 angles are evaluated in three parts with overlapped copies: grad_psi is bit for bit
    the device call's (each angle's planes are independent); T, hence grad_q, and the loss
    sum the parts in another order, so they agree to rounding."""
    pr = make_problem(64, 128, 12, seed=7)
    h = make_holo(pr)
    loss_d, gp_d, gq_d = h.gradient(dev(pr["psi"], torch.complex64))
    for _ in range(2):
        loss_h, gp_h, gq_h = h.gradient_host(pr["psi"].astype(np.complex64),
                                             sqrt_d=pr["sqrt_d"].astype(np.float32),
                                             q=pr["q"].astype(np.complex64))
        np.testing.assert_array_equal(gp_h, gp_d.cpu().numpy())
        assert abs(loss_h - loss_d) <= 1e-12 * abs(loss_d)
        assert rel(gq_h, gq_d.cpu().numpy()) < 1e-6
    F, _, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"], pr["geo"])
    assert abs(loss_h - F) / F < LOSS_TOL
    assert rel(gq_h, gq_ref) < GRAD_TOL


@pytest.mark.parametrize("functional", ["amplitude", "intensity"])
def test_gradient_host_chunks_in_parts(functional):
    """16 angles in two host calls of 8 (k0 = 0 with the reference term, k0 = 8 without),
    each run in parts: grad_psi slices are the device calls' bit for bit, and loss and grad_q
    summed over the calls match the device evaluation of all 16 angles to rounding (F1 and
    F2)."""
    pr = make_problem(64, 128, 16, seed=21)
    f1 = functional == "intensity"
    d = pr["sqrt_d"] ** 2 if f1 else pr["sqrt_d"]
    dref = pr["sqrt_dref"] ** 2 if f1 else pr["sqrt_dref"]
    from paper_2407_20304_gb300 import Holo
    geo = pr["geo"]
    h = Holo(geo.n, 16, geo.n_dist, geo.wavelength, geo.pixel, geo.Z, geo.z, pad=geo.P, chunk=8,
             w_ref=geo.w_ref, ext=geo.ext)
    h.set_functional(functional)
    h.set_shifts(pr["t"].astype(np.float32))
    h.set_data(dev(d, torch.float32), dev(dref, torch.float32))
    h.set_probe(dev(pr["q"], torch.complex64))
    psi = dev(pr["psi"], torch.complex64)
    gp_d = torch.empty_like(psi)
    gq_d = torch.empty((geo.P, geo.P), dtype=torch.complex64, device="cuda")
    loss_d = 0.0
    for i, k0 in enumerate((0, 8)):
        loss_d, _, _ = h.gradient(psi[k0:k0 + 8], grad_psi=gp_d[k0:k0 + 8], grad_q=gq_d, k0=k0,
                                  accumulate_q=i > 0, loss_in=loss_d)
    loss_h, gq_h = 0.0, np.zeros((geo.P, geo.P), np.complex64)
    for k0 in (0, 8):
        l, gp_h, g = h.gradient_host(pr["psi"][k0:k0 + 8].astype(np.complex64),
                                     sqrt_d=np.ascontiguousarray(d[k0:k0 + 8]).astype(np.float32),
                                     q=pr["q"].astype(np.complex64), k0=k0)
        np.testing.assert_array_equal(gp_h, gp_d[k0:k0 + 8].cpu().numpy())
        loss_h += l
        gq_h += g
    assert abs(loss_h - loss_d) <= 1e-6 * abs(loss_d)
    assert rel(gq_h, gq_d.cpu().numpy()) < 1e-5
    ref = (oh.gradients_f1 if f1 else oh.gradients)(pr["psi"], pr["q"], pr["t"], d, dref, geo)
    assert abs(loss_h - ref[0]) / ref[0] < LOSS_TOL
    assert rel(gq_h, ref[2]) < GRAD_TOL


def test_zero_gradient_at_noiseless_truth():
    pr = make_problem(64, 128, 2, seed=21, noiseless=True)
    h = make_holo(pr)
    h.set_probe(dev(pr["q_true"].astype(np.complex64), torch.complex64))
    psi_t = pr["psi_true"].astype(np.complex64)
    loss, gp, gq = h.gradient(dev(psi_t, torch.complex64))
    loss1, gp1, gq1 = h.gradient(dev(np.ones_like(psi_t), torch.complex64))
    assert loss < 1e-6 * loss1
    assert np.linalg.norm(gp.cpu().numpy()) < 1e-3 * np.linalg.norm(gp1.cpu().numpy())


def test_deterministic_repeat():
    pr = make_problem(64, 128, 3, seed=8)
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    a = h.gradient(psi)
    b = h.gradient(psi)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


# ------------------------------------------------------------------ CG vector ops

def test_dot_step_direction():
    from paper_2407_20304_gb300 import Holo
    h = Holo(16, 1, 1, G["wavelength"], G["pixel"], G["Z"], G["z"][:1], pad=32)
    rng = np.random.default_rng(3)
    for n in (1, 1000, 123457):
        a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
        b = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
        ref = np.real(np.vdot(a.astype(np.complex128), b.astype(np.complex128)))
        got = h.dot(dev(a, torch.complex64), dev(b, torch.complex64))
        assert abs(got - ref) <= 1e-5 * np.sqrt(n) * (abs(ref) + 1)
        x = dev(a, torch.complex64)
        h.step(x, dev(b, torch.complex64), 0.37)
        np.testing.assert_allclose(x.cpu().numpy(), a + np.float32(0.37) * b, rtol=1e-6, atol=1e-6)
        e = dev(a, torch.complex64)
        h.direction(e, dev(b, torch.complex64), -1.5)
        np.testing.assert_allclose(e.cpu().numpy(), -b + np.float32(-1.5) * a, rtol=1e-6, atol=1e-6)


def test_dy_dots_and_fused_direction_step():
    """One-pass DY inner products against FP64 NumPy and against the oracle's beta; the
    fused direction + step equals holo_direction then holo_step bit for bit."""
    from paper_2407_20304_gb300 import Holo
    from oracle import cg as ocg
    h = Holo(16, 1, 1, G["wavelength"], G["pixel"], G["Z"], G["z"][:1], pad=32)
    rng = np.random.default_rng(5)
    for n in (1, 4097, 300001):
        g, gp, eta, x = [(rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
                         for _ in range(4)]
        got = h.dy_dots(dev(g, torch.complex64), dev(gp, torch.complex64), dev(eta, torch.complex64))
        c = lambda u: u.astype(np.complex128)
        ref = (np.real(np.vdot(c(g), c(g))), np.real(np.vdot(c(g), c(eta))),
               np.real(np.vdot(c(gp), c(eta))))
        for a_, b_ in zip(got, ref):
            assert abs(a_ - b_) <= 1e-5 * np.sqrt(n) * (abs(b_) + 1)
        beta_ref = ocg.dai_yuan_beta(c(g), c(gp), c(eta))
        den = got[1] - got[2]
        if abs(den) > 1e-3 * np.sqrt(n):
            assert (den > 0) == (beta_ref is not None)
        if den > 0 and beta_ref is not None:
            assert abs(got[0] / den - beta_ref) <= 1e-4 * abs(beta_ref) + 1e-12
        x1, e1 = dev(x, torch.complex64), dev(eta, torch.complex64)
        h.direction(e1, dev(g, torch.complex64), 0.63)
        h.step(x1, e1, -0.21)
        x2, e2 = dev(x, torch.complex64), dev(eta, torch.complex64)
        h.direction_step(x2, e2, dev(g, torch.complex64), 0.63, -0.21)
        assert torch.equal(x1, x2) and torch.equal(e1, e2)


@pytest.mark.parametrize("n,P,K,accumulate", [(64, 128, 3, False), (256, 512, 2, True),
                                                (2048, 4096, 1, False)])
def test_dy_products_formed_in_the_gradient_and_the_step(n, P, K, accumulate):
    """holo_set_dy_direction / holo_direction_step_dy / holo_read_dy: the Dai-Yuan products
    formed inside pass D and the direction step against FP64 NumPy of the same vectors, and
    against holo_dy_dots; the step's x and eta equal holo_direction_step's bit for bit."""
    pr = make_problem(n, P, K, J=2, seed=7 * n + K, point="object")
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    rng = np.random.default_rng(n)
    c64 = lambda a: dev(a.astype(np.complex64), torch.complex64)
    eta = c64(rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)))
    g_prev = c64(rng.standard_normal((K, n, n)) + 1j * rng.standard_normal((K, n, n)))
    g = torch.zeros_like(psi) if not accumulate else c64(0.1 * rng.standard_normal((K, n, n)))
    h.set_dy_direction(eta)
    gq = torch.zeros((P, P), dtype=torch.complex64, device="cuda")
    h.gradient(psi, grad_psi=g, grad_q=gq, accumulate=accumulate)
    gg, ge, _ = h.read_dy()
    c = lambda t: t.cpu().numpy().astype(np.complex128)
    ref_gg, ref_ge = np.real(np.vdot(c(g), c(g))), np.real(np.vdot(c(g), c(eta)))
    assert abs(gg - ref_gg) <= 1e-6 * ref_gg
    assert abs(ge - ref_ge) <= 1e-6 * np.sqrt(ref_gg * np.real(np.vdot(c(eta), c(eta))))
    d = h.dy_dots(g, g_prev, eta)
    assert abs(gg - d[0]) <= 1e-6 * d[0]
    # the step: x and eta as holo_direction_step, and Re <g, eta_new>
    x1, e1 = psi.clone(), eta.clone()
    h.direction_step(x1, e1, g, 0.37, -0.05)
    x2, e2 = psi.clone(), eta.clone()
    h.direction_step(x2, e2, g, 0.37, -0.05, dy=True)
    assert torch.equal(x1, x2) and torch.equal(e1, e2)
    _, _, gn = h.read_dy()
    ref_gn = np.real(np.vdot(c(g), c(e2)))
    assert abs(gn - ref_gn) <= 1e-6 * np.sqrt(ref_gg * np.real(np.vdot(c(e2), c(e2))))
    # cleared: a later gradient leaves the products of the last one
    h.set_dy_direction(None)
    h.gradient(psi, grad_psi=torch.empty_like(psi))
    assert h.read_dy()[0] == gg
    h.close()


def test_state_and_argument_errors():
    from paper_2407_20304_gb300 import Holo, HoloError
    h = Holo(32, 2, 2, G["wavelength"], G["pixel"], G["Z"], G["z"][:2], pad=64)
    psi = torch.ones((2, 32, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(HoloError, match="STATE"):
        h.gradient(psi)
    h.set_shifts(np.zeros((2, 2, 2), np.float32))
    with pytest.raises(HoloError, match="STATE"):
        h.forward(psi)
    with pytest.raises(HoloError, match="ARG"):
        h.set_shifts(np.full((2, 2, 2), np.nan, np.float32))
    assert h.lib.holo_set_functional(h.ctx, 7) == 1      # HOLO_ERR_ARG
    with pytest.raises(KeyError):
        h.set_functional("phase")


def test_set_data_copies_the_amplitudes():
    """holo_set_data copies the amplitudes (into the column pass's blocked layout): the
    caller may overwrite its buffer after the call without changing the results."""
    pr = make_problem(96, 192, 2, seed=23, point="object")
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    ref = h.gradient(psi)
    d = dev(pr["sqrt_d"], torch.float32)
    h.set_data(d, dev(pr["sqrt_dref"], torch.float32))
    d.fill_(7.0)
    again = h.gradient(psi)
    assert again[0] == ref[0]
    assert torch.equal(again[1], ref[1]) and torch.equal(again[2], ref[2])


def test_deferred_probe_gradient_matches_oracle():
    """Chunks with HOLO_DEFER_Q sum their probe-gradient sources (T and G'_j on the union
    boxes) and holo_finish_q propagates them once: grad_q matches the oracle and the
    per-chunk form to rounding, grad_psi and the loss are the per-chunk form's bit for bit; a
    forward call between the chunks (a line search) leaves the pending sources intact."""
    from paper_2407_20304_gb300 import HoloError
    pr = make_problem(64, 128, 5, seed=31, point="object")
    h = make_holo(pr, chunk=2)
    psi = dev(pr["psi"], torch.complex64)
    gp_a, gq_a = torch.empty_like(psi), torch.empty((128, 128), dtype=torch.complex64, device="cuda")
    gp_b = torch.empty_like(psi)
    loss_a = loss_b = 0.0
    for i, k0 in enumerate(range(0, 5, 2)):
        nk = min(2, 5 - k0)
        loss_a, _, _ = h.gradient(psi[k0:k0 + nk], grad_psi=gp_a[k0:k0 + nk], grad_q=gq_a, k0=k0,
                                  accumulate_q=i > 0, loss_in=loss_a)
    with pytest.raises(HoloError, match="STATE"):
        h.finish_q()
    for i, k0 in enumerate(range(0, 5, 2)):
        nk = min(2, 5 - k0)
        loss_b, _, none = h.gradient(psi[k0:k0 + nk], grad_psi=gp_b[k0:k0 + nk], k0=k0,
                                     accumulate_q=i > 0, loss_in=loss_b, defer_q=True)
        assert none is None
        h.forward(psi[0:2], k0=0)
    gq_b = h.finish_q()
    assert loss_b == loss_a and torch.equal(gp_b, gp_a)
    assert rel(gq_b.cpu().numpy(), gq_a.cpu().numpy()) < 1e-6
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"])
    assert abs(loss_b - F) / F < LOSS_TOL
    assert rel(gq_b.cpu().numpy(), gq_ref) < GRAD_TOL
    # finish_q adds with accumulate, and the sources are consumed
    with pytest.raises(HoloError, match="STATE"):
        h.finish_q()
    # the host-buffer call does not defer (rejected before any other check)
    from paper_2407_20304_gb300 import _lib
    host = np.zeros((2, 64, 64), np.complex64)
    out_q = np.zeros((128, 128), np.complex64)
    st = h.lib.holo_gradient_host(h.ctx, 0, 2, host.ctypes.data, None, None, None,
                                  host.ctypes.data, out_q.ctypes.data, _lib.DEFER_Q)
    assert st == 1
