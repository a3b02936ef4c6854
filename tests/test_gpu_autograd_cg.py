"""The autograd Function and the DY-CG driver, on the GPU through the C ABI.

* HoloLoss gives the oracle's F2 and gradients (both modes: gradients kept from the
  forward pass, or recomputed in backward).
* At the differentiation workload's size (psi 1024^2 on 2048^2, 90 angles, 4 distances)
  the gradients agree with central finite differences of the library's own F2
  (step 1e-3 relative, 64 random directions).
* The CG driver's iterates follow the FP64 oracle's driver (same line-search decisions,
  F within FP32 rounding) and F never increases.
"""

import numpy as np
import pytest

import holo_synth as hs
from oracle import cg as ocg
from oracle import holo as oh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


def small_problem(n=64, P=128, K=3, seed=2):
    rng = hs.rng_for(hs.SEED_BASE + 9, seed)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    w = hs.Workload("t", n, P, K, 4, "ellipses", n * 40.0 / 128, 0.0, K, seed)
    psi_true = hs.object_stack(w, range(K), rng)
    q_true = hs.striped_probe(P, n * 40.0 / 128, rng)
    t = hs.sample_shifts(K, 4, rng).astype(np.float32).astype(np.float64)
    sqrt_d = np.abs(oh.forward(psi_true, q_true, t, geo)).astype(np.float32)
    sqrt_dref = np.abs(oh.reference_field(q_true, geo)).astype(np.float32)
    psi0 = np.ones((K, n, n), np.complex64)
    q0 = hs.perturbed_probe(q_true, rng).astype(np.complex64)
    return geo, t, sqrt_d, sqrt_dref, psi0, q0


def make_holo(geo, K, t, sqrt_d, sqrt_dref, chunk=0):
    from paper_2407_20304_gb300 import Holo
    h = Holo(geo.n, K, 4, geo.wavelength, geo.pixel, geo.Z, geo.z, pad=geo.P, chunk=chunk)
    h.set_shifts(t.astype(np.float32))
    h.set_data(torch.from_numpy(sqrt_d).cuda(), torch.from_numpy(sqrt_dref).cuda())
    return h


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("recompute", [False, True])
def test_autograd_function_matches_oracle(recompute):
    from paper_2407_20304_gb300.autograd import holo_loss
    geo, t, sqrt_d, sqrt_dref, psi0, q0 = small_problem()
    h = make_holo(geo, 3, t, sqrt_d, sqrt_dref)
    psi = torch.from_numpy(psi0).cuda().requires_grad_(True)
    q = torch.from_numpy(q0).cuda().requires_grad_(True)
    loss = holo_loss(psi, q, h, recompute=recompute)
    (3.0 * loss).backward()
    F, gp, gq = oh.gradients(psi0.astype(np.complex128), q0.astype(np.complex128), t,
                             sqrt_d.astype(np.float64), sqrt_dref.astype(np.float64), geo)
    assert abs(loss.item() - F) / F < 1e-5
    assert rel(psi.grad.cpu().numpy() / 3.0, gp) < 1e-4
    assert rel(q.grad.cpu().numpy() / 3.0, gq) < 1e-4


@pytest.fixture(scope="module")
def diff_problem():
    """The differentiation workload: psi 1024^2 (layered phantom) on 2048^2, 90 angles x 4
    distances, striped probe, positive Poisson amplitudes of the workload's counts."""
    w = hs.workloads()["autograd"]
    n, P, K, J = w.n, w.P, w.n_angles, w.n_dist
    rng = hs.rng_for(w.seed, 0)
    t = hs.sample_shifts(K, J, rng).astype(np.float32)
    # positive amplitudes with the workload's count statistics (no method arithmetic)
    base = np.abs(hs.striped_probe(n, w.probe_sigma, rng)).astype(np.float32) + 0.2
    sqrt_d = np.ascontiguousarray(np.broadcast_to(base, (K, J, n, n)))
    sqrt_d = hs.poisson_amplitude(sqrt_d.astype(np.float64) ** 2, w.counts, rng).astype(np.float32)
    sqrt_dref = base
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    psi = hs.object_stack(w, range(K), rng).astype(np.complex64)
    q = hs.striped_probe(P, w.probe_sigma, rng).astype(np.complex64)
    return dict(w=w, t=t, sqrt_d=sqrt_d, sqrt_dref=sqrt_dref, geo=geo, psi=psi, q=q)


def test_autograd_matches_oracle_at_differentiation_size(diff_problem):
    """HoloLoss at the differentiation workload's size against the FP64 oracle: psi.grad of
    three sampled angles of the 90-angle evaluation against the oracle's per-plane terms (an
    angle's gradient depends only on its own planes), and F2, psi.grad and q.grad of a 2-angle
    problem (reference term included) against the oracle's full gradients."""
    from paper_2407_20304_gb300.autograd import holo_loss
    pr = diff_problem
    geo, t, d, dr = pr["geo"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"]
    t64, d64, dr64 = t.astype(np.float64), d.astype(np.float64), dr.astype(np.float64)
    q64 = pr["q"].astype(np.complex128)
    K = pr["psi"].shape[0]
    h = make_holo(geo, K, t, d, dr)
    psi = torch.from_numpy(pr["psi"]).cuda().requires_grad_(True)
    q = torch.from_numpy(pr["q"]).cuda().requires_grad_(True)
    holo_loss(psi, q, h).backward()
    gp = psi.grad.cpu().numpy()
    h.close()
    for k in (0, 45, 89):
        ref = sum(oh.plane_gradient(pr["psi"][k].astype(np.complex128), q64, t64[k][j], d64[k, j],
                                    geo, j)[1] for j in range(4))
        e = rel(gp[k].astype(np.complex128), ref)
        print(f"angle {k}: grad_psi relative L2 error {e:.2e}")
        assert e < 1e-4
    ks = [0, 45]
    h2 = make_holo(geo, 2, np.ascontiguousarray(t[ks]), np.ascontiguousarray(d[ks]), dr)
    psi2 = torch.from_numpy(np.ascontiguousarray(pr["psi"][ks])).cuda().requires_grad_(True)
    q2 = torch.from_numpy(pr["q"]).cuda().requires_grad_(True)
    loss = holo_loss(psi2, q2, h2, recompute=True)
    loss.backward()
    F, gp_ref, gq_ref = oh.gradients(pr["psi"][ks].astype(np.complex128), q64, t64[ks], d64[ks],
                                     dr64, geo)
    e = (abs(loss.item() - F) / F, rel(psi2.grad.cpu().numpy(), gp_ref),
         rel(q2.grad.cpu().numpy(), gq_ref))
    print(f"2-angle problem: loss {e[0]:.2e}, grad_psi {e[1]:.2e}, grad_q {e[2]:.2e}")
    assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4
    h2.close()


def test_autograd_finite_differences_at_differentiation_size(diff_problem):
    from paper_2407_20304_gb300.autograd import holo_loss
    pr = diff_problem
    K = pr["psi"].shape[0]
    h = make_holo(pr["geo"], K, pr["t"], pr["sqrt_d"], pr["sqrt_dref"])
    psi = torch.from_numpy(pr["psi"]).cuda()
    q = torch.from_numpy(pr["q"]).cuda()
    psi.requires_grad_(True)
    q.requires_grad_(True)
    loss = holo_loss(psi, q, h)
    loss.backward()
    gp, gq = psi.grad.detach(), q.grad.detach()
    gen = torch.Generator(device="cuda").manual_seed(5)
    errs = []
    with torch.no_grad():
        for _ in range(64):
            hp = torch.randn(psi.shape, dtype=torch.complex64, device="cuda", generator=gen)
            hq = torch.randn(q.shape, dtype=torch.complex64, device="cuda", generator=gen)
            hp *= psi.norm() / hp.norm()
            hq *= q.norm() / hq.norm()
            eps = 1e-3
            fp = holo_loss(psi + eps * hp, q + eps * hq, h).item()
            fm = holo_loss(psi - eps * hp, q - eps * hq, h).item()
            fd = (fp - fm) / (2 * eps)
            an = float((torch.real(torch.vdot(gp.flatten(), hp.flatten()))
                        + torch.real(torch.vdot(gq.flatten(), hq.flatten()))).item())
            errs.append(abs(fd - an) / max(abs(an), 1e-30))
    print(f"\nFD relative errors: median {np.median(errs):.2e}, max {np.max(errs):.2e}")
    assert np.median(errs) < 2e-3 and np.max(errs) < 2e-2


@pytest.mark.parametrize("rule,line_search", [("dai-yuan", "backtracking"),
                                              ("fletcher-reeves", "armijo"),
                                              ("polak-ribiere", "backtracking"),
                                              ("dai-yuan", "armijo")])
def test_cg_driver_follows_the_oracle_driver(rule, line_search):
    """Same decisions as the FP64 driver until one falls within FP32 rounding of a tie;
    F never increases.  Where the two drivers first choose different steps, the FP64
    driver's accepted step must have changed F by less than FP32 can resolve."""
    from paper_2407_20304_gb300.cg import Reconstruction
    geo, t, sqrt_d, sqrt_dref, psi0, q0 = small_problem(K=4, seed=4)
    h = make_holo(geo, 4, t, sqrt_d, sqrt_dref, chunk=3)
    rec = Reconstruction(h, torch.from_numpy(psi0).cuda(), torch.from_numpy(q0).cuda(),
                         rule=rule, line_search=line_search)
    iters = 4
    hist = rec.run(iters)
    ref = ocg.reconstruct(psi0.astype(np.complex128), q0.astype(np.complex128), t,
                          sqrt_d.astype(np.float64), sqrt_dref.astype(np.float64), geo, iters=iters,
                          rule=rule, line_search=line_search)
    F = np.array(hist["F"])
    Fo = np.array(ref["hist"]["F"])
    print("\nF gpu", F, "\nF oracle", Fo, "\ngamma psi", hist["gamma_psi"],
          ref["hist"]["gamma_psi"], "\ngamma q", hist["gamma_q"], ref["hist"]["gamma_q"])
    assert np.all(np.diff(F) <= 0)
    assert abs(F[0] - Fo[0]) / Fo[0] < 1e-5
    same = 0
    while (same < iters and hist["gamma_psi"][same] == ref["hist"]["gamma_psi"][same]
           and hist["gamma_q"][same] == ref["hist"]["gamma_q"][same]):
        same += 1
    assert same >= 1
    np.testing.assert_allclose(F[:same + 1], Fo[:same + 1], rtol=1e-4)
    if same < iters:
        # first differing decision: a near-tie for the block whose step differs
        # (whichever driver accepted the contested trial step saw F barely change)
        start = Fo[same]
        if hist["gamma_psi"][same] != ref["hist"]["gamma_psi"][same]:
            change = min(abs(start - ref["hist"]["F_after_psi"][same]),
                         abs(start - hist["F_after_psi"][same])) / start
        else:
            change = min(abs(ref["hist"]["F_after_psi"][same] - Fo[same + 1]),
                         abs(hist["F_after_psi"][same] - F[same + 1])) / start
        print("first different step at iteration", same, "relative change", change)
        assert change < 1e-4


@pytest.mark.parametrize("rule,line_search", [("dai-yuan", "backtracking"),
                                              ("fletcher-reeves", "armijo"),
                                              ("polak-ribiere", "backtracking"),
                                              ("dai-yuan", "armijo")])
def test_every_cg_iteration_matches_an_fp64_step_from_the_same_state(rule, line_search):
    """Pins every iteration, not only those before the first difference: before each GPU
    iteration the driver's state (psi, q, directions, gradients, trial steps) is handed to
    the FP64 oracle, which takes one iteration from it with the oracle's functional, line
    search and direction rule.  The accepted step lengths must be the GPU's, unless the
    oracle's accepted trial changed F by less than FP32 resolves (a near-tie, relative change
    < 1e-4); the new directions' beta must agree to 1e-4 relative."""
    from paper_2407_20304_gb300.cg import Reconstruction
    geo, t, sqrt_d, sqrt_dref, psi0, q0 = small_problem(K=4, seed=4)
    h = make_holo(geo, 4, t, sqrt_d, sqrt_dref, chunk=3)
    rec = Reconstruction(h, torch.from_numpy(psi0).cuda(), torch.from_numpy(q0).cuda(),
                         rule=rule, line_search=line_search)
    d64, r64 = sqrt_d.astype(np.float64), sqrt_dref.astype(np.float64)
    c = lambda x: x.detach().cpu().numpy().astype(np.complex128)
    rec.run(0)
    ties = 0
    for it in range(6):
        psi, q = c(rec.psi), c(rec.q)
        eta, g = [c(e) for e in rec.eta], [c(x) for x in rec.g]
        trial = list(rec.trial)
        F0 = oh.functional(psi, q, t, d64, r64, geo)

        def search(f, F, gb, x, e, tr):
            if line_search == "armijo":
                return ocg.armijo(f, F, ocg.re_inner(gb, e), x, e, tr, rec.max_halvings)
            return ocg.backtrack(f, F, x, e, tr, rec.max_halvings)

        gp_o, Fp = search(lambda x: oh.functional(x, q, t, d64, r64, geo), F0, g[0], psi, eta[0],
                          trial[0])
        psi_o = psi + gp_o * eta[0]
        gq_o, Fq = search(lambda x: oh.functional(psi_o, x, t, d64, r64, geo), Fp, g[1], q,
                          eta[1], trial[1])
        rec.run(1)
        hist = rec.history
        for name, mine, theirs, before, after in (("psi", hist["gamma_psi"][-1], gp_o, F0, Fp),
                                                  ("q", hist["gamma_q"][-1], gq_o, Fp, Fq)):
            if mine != theirs:
                change = abs(before - after) / before
                print(f"iteration {it}: {name} step {mine} (gpu) vs {theirs} (fp64), "
                      f"relative F change of the fp64 step {change:.1e}")
                assert change < 1e-4
                ties += 1
        if hist["gamma_psi"][-1] != gp_o or hist["gamma_q"][-1] != gq_o:
            continue
        # the direction update from the GPU's new gradients, in FP64
        g_new = [c(x) for x in rec.g]
        for b, key in ((0, "beta_psi"), (1, "beta_q")):
            _, beta_o = ocg.direction(g_new[b], g[b], eta[b], rule)
            beta = hist[key][-1]
            assert abs(beta - beta_o) <= 1e-4 * max(abs(beta_o), 1e-12) or \
                (beta == 0.0) == (beta_o == 0.0) == True, (it, key, beta, beta_o)
    assert ties <= 2


@pytest.mark.parametrize("n,P", [(64, 128), (48, 96), (256, 512)])
def test_initial_probe_matches_oracle(n, P):
    """The paper's initial probe (reference image propagated back to plane 0) against the
    oracle's initial_probe."""
    from paper_2407_20304_gb300 import Holo
    rng = np.random.default_rng(n)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    a = (1.0 + 0.3 * rng.standard_normal((n, n))).astype(np.float32)
    h = Holo(n, 1, 4, geo.wavelength, geo.pixel, geo.Z, geo.z, pad=P)
    got = h.initial_probe(torch.from_numpy(a).cuda()).cpu().numpy()
    ref = oh.initial_probe(a.astype(np.float64), geo)
    assert rel(got.astype(np.complex128), ref) < 1e-5
