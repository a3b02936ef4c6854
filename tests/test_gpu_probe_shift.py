"""Probe shifts s_kj (Eq. min1 / Eq. min2) on the CUDA path, against the FP64 oracle.

With probe shifts the library runs the SHIFT forms of passes A-C on the whole padded grid
(the shift moved off the probe onto the detector-side propagation and the object shift
t - m~ s).  Tolerances as in test_gpu_parity.py: loss 1e-5, gradients 1e-4 (relative L2).
Data are made by the oracle, never by the CUDA path.
"""

import numpy as np
import pytest

import evalpoints as ep
import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY
LOSS_TOL, GRAD_TOL = 1e-5, 1e-4


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


def make_problem(n, P, K, J=4, ext=1.0, w_ref=1.0, seed=0, smax=2.0, point="start"):
    """point: "start" (psi = 1 for ext = 1), "iterated" (5 oracle CG iterations from the
    start point, probe shifts included) or "object" (the perturbed true object)."""
    rng = hs.rng_for(hs.SEED_BASE + 11, seed)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], tuple(G["z"][:J]), n, P, ext=ext,
                      w_ref=w_ref)
    w = hs.Workload("t", n, P, K, J, "ellipses", n * 40.0 / 128, 0.0, K, seed)
    psi_true = hs.object_stack(w, range(K), rng)
    q_true = hs.striped_probe(P, n * 40.0 / 128, rng)
    t = hs.sample_shifts(K, J, rng).astype(np.float32).astype(np.float64)
    s = rng.uniform(-smax, smax, (K, J, 2)).astype(np.float32).astype(np.float64)
    sqrt_d = np.abs(oh.forward(psi_true, q_true, t, geo, probe_shifts=s))
    sqrt_dref = np.abs(oh.reference_field(q_true, geo))
    sqrt_d = hs.poisson_amplitude(sqrt_d ** 2, 1e4, rng).astype(np.float32).astype(np.float64)
    sqrt_dref = hs.poisson_amplitude(sqrt_dref ** 2, 1e4, rng).astype(np.float32).astype(np.float64)
    psi0 = np.ones((K, n, n), np.complex128) if ext == 1.0 else hs.transmittance(
        -0.5 * rng.uniform(0, 1, (K, n, n))).astype(np.complex64).astype(np.complex128)
    q0 = hs.perturbed_probe(q_true, rng).astype(np.complex64).astype(np.complex128)
    if point == "iterated":
        psi0, q0 = ep.iterated_point(psi0, q0, t, sqrt_d, sqrt_dref, geo, probe_shifts=s)
    elif point == "object":
        psi0 = ep.object_point(psi_true, rng)
    return dict(geo=geo, psi=psi0, q=q0, t=t, s=s, sqrt_d=sqrt_d, sqrt_dref=sqrt_dref)


def make_holo(pr, chunk=0, probe_shifts=True, functional="amplitude"):
    from paper_2407_20304_gb300 import Holo
    geo = pr["geo"]
    K = pr["psi"].shape[0]
    h = Holo(geo.n, K, geo.n_dist, geo.wavelength, geo.pixel, geo.Z, geo.z, pad=geo.P,
             chunk=chunk, w_ref=geo.w_ref, ext=geo.ext)
    h.set_functional(functional)
    if probe_shifts:
        h.set_probe_shifts(pr["s"].astype(np.float32))
    h.set_shifts(pr["t"].astype(np.float32))
    f1 = functional == "intensity"
    d = pr["sqrt_d"] ** 2 if f1 else pr["sqrt_d"]
    dref = pr["sqrt_dref"] ** 2 if f1 else pr["sqrt_dref"]
    h.set_data(dev(d, torch.float32), dev(dref, torch.float32) if geo.w_ref else None)
    h.set_probe(dev(pr["q"], torch.complex64))
    return h


@pytest.mark.parametrize("n,P,K,J,ext,w_ref", [
    (16, 32, 2, 4, 1.0, 1.0), (32, 64, 3, 4, 1.0, 1.0), (32, 64, 2, 4, 0.0, 0.0),
    (100, 256, 2, 3, 1.0, 0.0), (128, 256, 3, 4, 1.0, 1.0), (256, 512, 2, 4, 1.0, 1.0),
    # radix-3 line lengths
    (48, 96, 2, 4, 1.0, 1.0), (384, 768, 1, 4, 1.0, 1.0),
    # plane-split pass B (n <= 1024) and whole column-group rounds (n = 1826, 2048)
    (512, 1024, 2, 4, 1.0, 1.0), (1826, 2048, 1, 2, 1.0, 1.0), (2048, 4096, 1, 2, 1.0, 1.0),
])
def test_probe_shift_gradient_matches_oracle(n, P, K, J, ext, w_ref):
    pr = make_problem(n, P, K, J=J, ext=ext, w_ref=w_ref, seed=7 * n + J)
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    loss_f = h.forward(psi)
    loss, gp, gq = h.gradient(psi)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"], probe_shifts=pr["s"])
    assert abs(loss_f - F) / F < LOSS_TOL
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL


@pytest.mark.parametrize("n,P,K,J,point", [
    (32, 64, 2, 4, "iterated"), (48, 96, 2, 4, "iterated"), (128, 256, 2, 4, "iterated"),
    (384, 768, 1, 4, "object"), (512, 1024, 2, 4, "object"), (1826, 2048, 1, 2, "object"),
    (2048, 4096, 1, 2, "object"),
])
def test_probe_shift_gradient_away_from_start(n, P, K, J, point):
    """Production mode (ext = 1) with probe shifts away from psi = 1: the full-grid gather of
    R' psi at the object shift t - m~ s and the conj(R' psi) v term of the probe gradient."""
    pr = make_problem(n, P, K, J=J, seed=17 * n + J, point=point)
    assert np.abs(pr["psi"] - 1).mean() > 1e-2
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64)
    loss_f = h.forward(psi)
    loss, gp, gq = h.gradient(psi)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"], probe_shifts=pr["s"])
    assert abs(loss_f - F) / F < LOSS_TOL
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL


def test_probe_shift_fields_match_oracle():
    pr = make_problem(64, 128, 2, seed=3)
    h = make_holo(pr)
    u = torch.empty((2, 4, 64, 64), dtype=torch.complex64, device="cuda")
    h.forward(dev(pr["psi"], torch.complex64), u_out=u)
    u_ref = oh.forward(pr["psi"], pr["q"], pr["t"], pr["geo"], probe_shifts=pr["s"])
    assert rel(u.cpu().numpy(), u_ref) < 1e-5


def test_probe_shift_intensity_functional():
    pr = make_problem(64, 128, 2, seed=4)
    h = make_holo(pr, functional="intensity")
    loss, gp, gq = h.gradient(dev(pr["psi"], torch.complex64))
    F, gp_ref, gq_ref = oh.gradients_f1(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"] ** 2,
                                        pr["sqrt_dref"] ** 2, pr["geo"], probe_shifts=pr["s"])
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL


def test_zero_probe_shifts_match_the_box_form_and_clearing_restores_it():
    """Zero probe shifts run the full-grid form, which must agree with the box form to
    rounding; clearing the shifts gives the box form's results bit for bit."""
    pr = make_problem(64, 128, 3, seed=5)
    psi = dev(pr["psi"], torch.complex64)
    hb = make_holo(pr, probe_shifts=False)
    lb, gpb, gqb = hb.gradient(psi)
    hz = make_holo(pr, probe_shifts=False)
    hz.set_probe_shifts(np.zeros((3, 4, 2), np.float32))
    lz, gpz, gqz = hz.gradient(psi)
    assert abs(lz - lb) / lb < 1e-6
    assert rel(gpz.cpu().numpy(), gpb.cpu().numpy()) < 1e-5
    assert rel(gqz.cpu().numpy(), gqb.cpu().numpy()) < 1e-5
    hz.set_probe_shifts(None)
    lc, gpc, gqc = hz.gradient(psi)
    assert lc == lb
    assert torch.equal(gpc, gpb) and torch.equal(gqc, gqb)


def test_probe_shift_chunks_and_host_call():
    """Chunked device calls and the host-buffer call (in parts) agree with the oracle under
    probe shifts; the host call's grad_psi is the device call's bit for bit."""
    pr = make_problem(64, 128, 8, seed=6)
    h = make_holo(pr, chunk=4)
    psi = dev(pr["psi"], torch.complex64)
    gp = torch.empty_like(psi)
    gq = torch.empty((128, 128), dtype=torch.complex64, device="cuda")
    loss = 0.0
    for i, k0 in enumerate((0, 4)):
        loss, _, _ = h.gradient(psi[k0:k0 + 4], grad_psi=gp[k0:k0 + 4], grad_q=gq, k0=k0,
                                accumulate_q=i > 0, loss_in=loss)
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"], probe_shifts=pr["s"])
    assert abs(loss - F) / F < LOSS_TOL
    assert rel(gp.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(gq.cpu().numpy(), gq_ref) < GRAD_TOL
    lh, gqh = 0.0, np.zeros((128, 128), np.complex64)
    for k0 in (0, 4):
        l, gph, g = h.gradient_host(pr["psi"][k0:k0 + 4].astype(np.complex64),
                                    sqrt_d=pr["sqrt_d"][k0:k0 + 4].astype(np.float32),
                                    q=pr["q"].astype(np.complex64), k0=k0)
        np.testing.assert_array_equal(gph, gp[k0:k0 + 4].cpu().numpy())
        lh += l
        gqh += g
    assert abs(lh - loss) <= 1e-6 * abs(loss)
    assert rel(gqh, gq.cpu().numpy()) < 1e-5


def test_probe_shift_argument_errors():
    from paper_2407_20304_gb300 import HoloError
    pr = make_problem(32, 64, 2, seed=8)
    h = make_holo(pr, probe_shifts=False)
    bad = np.zeros((2, 4, 2), np.float32)
    bad[1, 2, 0] = 17.0  # > n/2
    with pytest.raises(HoloError):
        h.set_probe_shifts(bad)
    bad[1, 2, 0] = np.nan
    with pytest.raises(HoloError):
        h.set_probe_shifts(bad)
    with pytest.raises(ValueError):
        h.set_probe_shifts(np.zeros((2, 3, 2), np.float32))


@pytest.mark.parametrize("recompute", [False, True])
def test_probe_shift_autograd(recompute):
    """The autograd Function on a context with probe shifts: loss and .grad against the
    oracle (both stored-gradient and recompute modes)."""
    from paper_2407_20304_gb300.autograd import holo_loss
    pr = make_problem(64, 128, 2, seed=9)
    h = make_holo(pr)
    psi = dev(pr["psi"], torch.complex64).requires_grad_(True)
    q = dev(pr["q"], torch.complex64).requires_grad_(True)
    loss = holo_loss(psi, q, h, recompute=recompute)
    loss.backward()
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"], probe_shifts=pr["s"])
    assert abs(loss.detach().item() - F) / F < LOSS_TOL
    assert rel(psi.grad.cpu().numpy(), gp_ref) < GRAD_TOL
    assert rel(q.grad.cpu().numpy(), gq_ref) < GRAD_TOL
