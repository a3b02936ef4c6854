"""Batched evaluation of uneven reconstructions: the captured graph (any schedule) gives
exactly the per-instance loop's results, and those match the FP64 oracle.  The instances mix
sides 32 .. 2048 (P = 64 .. 4096, including the radix-3 lengths 96 and 768) and evaluation
points: psi = 1 and the perturbed true object (where the object field is not zero)."""

import numpy as np
import pytest

import evalpoints as ep
import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY


def pad_of(n):
    return 2 * n        # 64, 96 (radix-3 step), 128


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_20304_gb300 import Holo
    from paper_2407_20304_gb300.batch import HoloBatch, Instance
    rng = hs.rng_for(hs.SEED_BASE + 3000, 0)
    specs = [(32, 3, 2), (48, 2, 4), (64, 5, 1), (32, 4, 3), (48, 3, 2), (64, 2, 4),
             (384, 1, 2), (2048, 1, 1)]
    insts, refs = [], []
    for i, (n, K, J) in enumerate(specs):
        P = pad_of(n)
        z = tuple(G["z"][:J])
        geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], z, n, P)
        w = hs.Workload("b", n, P, K, J, "ellipses", n / 3, 0.0, K, i)
        psi_true = hs.object_stack(w, range(K), rng)
        q_true = hs.striped_probe(P, n / 3, rng)
        t = hs.sample_shifts(K, J, rng).astype(np.float32).astype(np.float64)
        sqrt_d = np.abs(oh.forward(psi_true, q_true, t, geo)).astype(np.float32)
        sqrt_dref = np.abs(oh.reference_field(q_true, geo)).astype(np.float32)
        psi0 = (np.ones((K, n, n), np.complex128) if i % 2 == 0 and n < 256 else
                ep.object_point(psi_true, rng)).astype(np.complex64)
        q0 = hs.perturbed_probe(q_true, rng).astype(np.complex64)
        h = Holo(n, K, J, G["wavelength"], G["pixel"], G["Z"], z, pad=P, chunk=min(2, K))
        h.set_shifts(t.astype(np.float32))
        d, dr = torch.from_numpy(sqrt_d).cuda(), torch.from_numpy(sqrt_dref).cuda()
        h.set_data(d, dr)
        insts.append(Instance(h, torch.from_numpy(psi0).cuda(), torch.from_numpy(q0).cuda()))
        refs.append(oh.gradients(psi0.astype(np.complex128), q0.astype(np.complex128), t,
                                 sqrt_d.astype(np.float64), sqrt_dref.astype(np.float64), geo))
    return HoloBatch(insts), refs


def test_loop_matches_oracle(batch):
    b, refs = batch
    b.run_loop()
    torch.cuda.synchronize()
    for it, (F, gp, gq) in zip(b.inst, refs):
        assert abs(it.h.read_loss() - F) / F < 1e-5
        e_p = np.linalg.norm(it.grad_psi.cpu().numpy() - gp) / np.linalg.norm(gp)
        e_q = np.linalg.norm(it.grad_q.cpu().numpy() - gq) / np.linalg.norm(gq)
        assert e_p < 1e-4 and e_q < 1e-4


@pytest.mark.parametrize("branches", [1, 3])
def test_graph_replay_equals_loop(batch, branches):
    b, _ = batch
    b.run_loop()
    torch.cuda.synchronize()
    ref = [(it.h.read_loss(), it.grad_psi.clone(), it.grad_q.clone()) for it in b.inst]
    for it in b.inst:
        it.grad_psi.zero_()
        it.grad_q.zero_()
    cost = [float(it.planes) for it in b.inst]
    b.capture(b.balanced(branches, cost))
    b.replay()
    b.replay()
    torch.cuda.synchronize()
    for it, (F, gp, gq) in zip(b.inst, ref):
        assert it.h.read_loss() == F
        assert torch.equal(it.grad_psi, gp) and torch.equal(it.grad_q, gq)


def test_autotune_picks_a_schedule(batch):
    b, _ = batch
    ms, sched, cost = b.autotune(candidates=(1, 2, 4), reps=1)
    assert sorted(i for g in sched for i in g) == list(range(len(b.inst)))
    assert ms > 0 and len(b.tuning) >= 2


def _snapshot(b):
    torch.cuda.synchronize()
    return [(it.h.read_loss(), it.grad_psi.clone(), it.grad_q.clone()) for it in b.inst]


def _clear(b):
    for it in b.inst:
        it.grad_psi.fill_(float("nan"))
        it.grad_q.fill_(float("nan"))


def test_persistent_graph_equals_loop_and_oracle(batch):
    """The persistent form (passes A-D of all problems as multi-problem launches walking work
    lists, captured once, replayed twice) gives every problem the per-problem loop's loss,
    grad_psi and grad_q bit for bit (same schedule), and those match the FP64 oracle, at
    sides 32 .. 2048 including the radix-3 lengths."""
    b, refs = batch
    b.prepare_persistent()
    b.run_loop()
    ref = _snapshot(b)
    _clear(b)
    b.capture_persistent()
    b.replay_persistent()
    b.replay_persistent()
    got = _snapshot(b)
    for (F, gp, gq), (F2, gp2, gq2), (Fo, gpo, gqo) in zip(ref, got, refs):
        assert F2 == F
        assert torch.equal(gp2, gp) and torch.equal(gq2, gq)
        assert abs(F2 - Fo) / Fo < 1e-5
        assert np.linalg.norm(gp2.cpu().numpy() - gpo) / np.linalg.norm(gpo) < 1e-4
        assert np.linalg.norm(gq2.cpu().numpy() - gqo) / np.linalg.norm(gqo) < 1e-4


def test_persistent_autotune_keeps_the_results(batch):
    """The schedule autotuner changes only launch shapes: after it, the replayed persistent
    graph still equals the per-problem loop run with the chosen schedule."""
    b, _ = batch
    ms, chosen = b.autotune_persistent(reps=1)
    assert ms > 0 and set(chosen) == set(b.line_lengths()) and len(b.ptuning) >= 2
    b.run_loop()
    ref = _snapshot(b)
    _clear(b)
    b.replay_persistent()
    got = _snapshot(b)
    for (F, gp, gq), (F2, gp2, gq2) in zip(ref, got):
        assert F2 == F and torch.equal(gp2, gp) and torch.equal(gq2, gq)


@pytest.mark.parametrize("layout", ["per_length", "per_length_x2"])
def test_persistent_per_length_branches_equal_loop(batch, layout):
    """One (or two) library batches per line length, each on its own branch of the captured
    graph: still every problem's own results bit for bit."""
    b, _ = batch
    b.prepare_persistent(layout)
    assert len(b._pbs) >= len(b.line_lengths())
    b.run_loop()
    ref = _snapshot(b)
    _clear(b)
    b.capture_persistent()
    b.replay_persistent()
    got = _snapshot(b)
    for (F, gp, gq), (F2, gp2, gq2) in zip(ref, got):
        assert F2 == F and torch.equal(gp2, gp) and torch.equal(gq2, gq)
