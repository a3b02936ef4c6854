"""The unfused cuFFT comparison form computes the oracle's F2 and gradients (so the
benchmark compares like with like): batched over groups of planes, with a last group that is
not full, at the perturbed true object."""

import numpy as np
import pytest

import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY


def test_unfused_form_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import bench
    n, P, K = 64, 128, 3
    rng = hs.rng_for(hs.SEED_BASE + 13, 0)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    w = hs.Workload("t", n, P, K, 4, "ellipses", 20.0, 0.0, K, 0)
    psi_true = hs.object_stack(w, range(K), rng)
    q = hs.striped_probe(P, 20.0, rng).astype(np.complex64)
    t = hs.sample_shifts(K, 4, rng).astype(np.float32).astype(np.float64)
    sqrt_d = np.abs(oh.forward(psi_true, q.astype(np.complex128), t, geo)).astype(np.float32) * 0.9
    sqrt_dref = np.abs(oh.reference_field(q.astype(np.complex128), geo)).astype(np.float32)
    psi = hs.perturbed_probe(psi_true, rng, 0.05).astype(np.complex64)
    u = bench.Unfused(n, P, G, t, torch.from_numpy(sqrt_d).cuda(), torch.from_numpy(sqrt_dref).cuda(),
                      group=2)
    loss, gp, gq = u.gradient(torch.from_numpy(psi).cuda(), torch.from_numpy(q).cuda())
    loss = float(loss)
    F, gp_ref, gq_ref = oh.gradients(psi.astype(np.complex128), q.astype(np.complex128), t,
                                     sqrt_d.astype(np.float64), sqrt_dref.astype(np.float64), geo)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert abs(loss - F) / F < 1e-5
    assert rel(gp.cpu().numpy(), gp_ref) < 1e-4
    assert rel(gq.cpu().numpy(), gq_ref) < 1e-4
