"""Full-size parity: psi 2048^2 on the 4096^2 grid, 4 distances, against the FP64 oracle.

The benchmark's launch configuration (a 60-angle chunk) is evaluated on the GPU and the
gradients grad_psi_k of four sampled angles are compared with the oracle's per-plane terms
(grad_psi_k depends only on the planes of angle k).  The loss and grad_q, which sum over
every plane of a chunk, are compared on a 4-angle chunk of the same problem.  Relative L2
errors are printed (the precision report of FP32 wavefields with FP64 reductions).

Two evaluation points: the start point psi = 1 (where the object field R0(psi - 1) is zero)
and the layered phantom times a small perturbation (where pass A's gather of the object at
P = 4096 and the conj(w) v term of grad_q are exercised).
"""

import time

import numpy as np
import pytest

import evalpoints as ep
import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
LOSS_TOL, GRAD_TOL = 1e-5, 1e-4
SAMPLED = (0, 17, 38, 59)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    w = hs.workloads()["large"]
    g = hs.WORKLOAD_GEOMETRY
    n, P, K, J = w.n, w.P, w.chunk, w.n_dist
    rng = hs.rng_for(w.seed, 11)
    psi_true = hs.object_stack(w, range(K), rng)
    q_true = hs.striped_probe(P, w.probe_sigma, rng)
    t = hs.sample_shifts(K, J, rng).astype(np.float32).astype(np.float64)
    q0 = hs.perturbed_probe(q_true, rng).astype(np.complex64).astype(np.complex128)
    geo = oh.Geometry(g["wavelength"], g["pixel"], g["Z"], tuple(g["z"]), n, P)
    t0 = time.time()
    # data of the sampled angles by the oracle; the other angles get unrelated amplitudes
    sqrt_d = np.empty((K, J, n, n), np.float32)
    filler = np.abs(hs.striped_probe(n, n / 3, rng)).astype(np.float32) + 0.5
    sqrt_d[:] = filler
    u = oh.forward(psi_true[list(SAMPLED)], q_true, t[list(SAMPLED)], geo)
    amp = hs.poisson_amplitude(np.abs(u) ** 2, w.counts, rng).astype(np.float32)
    for s, k in enumerate(SAMPLED):
        sqrt_d[k] = amp[s]
    sqrt_dref = hs.poisson_amplitude(np.abs(oh.reference_field(q_true, geo)) ** 2, w.counts,
                                     rng).astype(np.float32)
    psis = {"start": np.ones((K, n, n), np.complex64),
            "object": psi_true.astype(np.complex64)}
    for k in SAMPLED:
        psis["object"][k] = ep.object_point(psi_true[k], rng)
    del psi_true
    # oracle per-plane terms of the sampled angles at both points (q = q0)
    terms = {}
    for point, psi in psis.items():
        for k in SAMPLED:
            for j in range(J):
                terms[(point, k, j)] = oh.plane_gradient(
                    psi[k].astype(np.complex128), q0, t[k][j], sqrt_d[k, j].astype(np.float64),
                    geo, j)
    print(f"\noracle set-up {time.time() - t0:.0f} s")
    return dict(w=w, g=g, n=n, P=P, K=K, J=J, t=t, q0=q0, sqrt_d=sqrt_d, sqrt_dref=sqrt_dref,
                psis=psis, terms=terms, geo=geo)


def _holo(pr, K, sqrt_d):
    from paper_2407_20304_gb300 import Holo
    g = pr["g"]
    h = Holo(pr["n"], K, pr["J"], g["wavelength"], g["pixel"], g["Z"], g["z"], pad=pr["P"])
    h.set_data(torch.from_numpy(sqrt_d).cuda(), torch.from_numpy(pr["sqrt_dref"]).cuda())
    h.set_probe(torch.from_numpy(pr["q0"].astype(np.complex64)).cuda())
    return h


@pytest.mark.parametrize("point", ["start", "object"])
def test_grad_psi_of_sampled_angles_in_the_benchmark_chunk(problem, point):
    pr = problem
    h = _holo(pr, pr["K"], pr["sqrt_d"])
    h.set_shifts(pr["t"].astype(np.float32))
    _, gp, _ = h.gradient(torch.from_numpy(pr["psis"][point]).cuda())
    gp = gp.cpu().numpy()
    for k in SAMPLED:
        ref = sum(pr["terms"][(point, k, j)][1] for j in range(pr["J"]))
        e = rel(gp[k].astype(np.complex128), ref)
        print(f"{point}, angle {k}: grad_psi relative L2 error {e:.2e}")
        assert e < GRAD_TOL
    h.close()


@pytest.mark.parametrize("point", ["start", "object"])
def test_loss_and_grad_q_on_a_four_angle_chunk(problem, point):
    pr = problem
    ks = list(SAMPLED)
    h = _holo(pr, 4, np.ascontiguousarray(pr["sqrt_d"][ks]))
    h.set_shifts(pr["t"][ks].astype(np.float32))
    loss, gp, gq = h.gradient(torch.from_numpy(np.ascontiguousarray(pr["psis"][point][ks])).cuda())
    geo, J = pr["geo"], pr["J"]
    d = oh.derived_geometry(geo.z, geo.Z)
    F = sum(pr["terms"][(point, k, j)][0] for k in ks for j in range(J))
    gq_ref = np.zeros((pr["P"], pr["P"]), np.complex128)
    for j in range(J):
        G = sum(pr["terms"][(point, k, j)][2] for k in ks)
        gq_ref += 2 * oh.propagate(G, -d["omega"][j], geo.wavelength, geo.pixel)
    uref = oh.reference_field(pr["q0"], geo)
    aref = pr["sqrt_dref"].astype(np.float64)
    F += float(np.sum((np.abs(uref) - aref) ** 2))
    gq_ref += 2 * oh.propagate(oh.embed(oh.amplitude_residual(uref, aref), pr["P"]), -d["zeta"][0],
                               geo.wavelength, geo.pixel)
    e_l = abs(loss - F) / F
    e_q = rel(gq.cpu().numpy().astype(np.complex128), gq_ref)
    e_p = max(rel(gp.cpu().numpy()[s].astype(np.complex128),
                  sum(pr["terms"][(point, k, j)][1] for j in range(J))) for s, k in enumerate(ks))
    print(f"{point}, 4-angle chunk: loss {e_l:.2e}, grad_q {e_q:.2e}, grad_psi (max over angles) {e_p:.2e}")
    assert e_l < LOSS_TOL and e_q < GRAD_TOL and e_p < GRAD_TOL
    h.close()


def test_intensity_functional_on_a_four_angle_chunk(problem):
    """F1 (Eq. min2) at full size: loss and both gradients of a 4-angle chunk against the
    oracle's gradients_f1 (intensities d = sqrt_d^2 as data)."""
    pr = problem
    ks = list(SAMPLED)
    d = np.ascontiguousarray(pr["sqrt_d"][ks]).astype(np.float64) ** 2
    dref = pr["sqrt_dref"].astype(np.float64) ** 2
    h = _holo(pr, 4, np.ascontiguousarray(pr["sqrt_d"][ks]))
    h.set_functional("intensity")
    h.set_data(torch.from_numpy(d.astype(np.float32)).cuda(), torch.from_numpy(dref.astype(np.float32)).cuda())
    h.set_shifts(pr["t"][ks].astype(np.float32))
    psi = np.ascontiguousarray(pr["psis"]["object"][ks])
    loss, gp, gq = h.gradient(torch.from_numpy(psi).cuda())
    F, gp_ref, gq_ref = oh.gradients_f1(psi.astype(np.complex128), pr["q0"], pr["t"][ks],
                                        d.astype(np.float32).astype(np.float64),
                                        dref.astype(np.float32).astype(np.float64), pr["geo"])
    e_l = abs(loss - F) / F
    e_p = rel(gp.cpu().numpy().astype(np.complex128), gp_ref)
    e_q = rel(gq.cpu().numpy().astype(np.complex128), gq_ref)
    print(f"F1 4-angle chunk: loss {e_l:.2e}, grad_psi {e_p:.2e}, grad_q {e_q:.2e}")
    assert e_l < LOSS_TOL and e_p < GRAD_TOL and e_q < GRAD_TOL
    h.close()
