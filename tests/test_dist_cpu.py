"""Shared-probe sharding over two ranks (gloo, CPU): the per-rank partial losses and probe
gradients, all-reduced, equal the full problem's; grad_psi shards are exact slices.  With and
without probe shifts s_kj (sliced with the angles like t_kj)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import holo_synth as hs
from oracle import holo as oh
from paper_2407_20304_gb300.dist import allreduce_loss_and_grad_q, shard

G = hs.WORKLOAD_GEOMETRY


def _problem(probe_shifts=False):
    n, P, K = 16, 32, 5
    rng = hs.rng_for(hs.SEED_BASE + 21, 0)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    w = hs.Workload("t", n, P, K, 4, "ellipses", 6.0, 0.0, K, 0)
    psi = hs.object_stack(w, range(K), rng)
    q = hs.striped_probe(P, 6.0, rng)
    t = hs.sample_shifts(K, 4, rng)
    s = rng.uniform(-2, 2, (K, 4, 2)) if probe_shifts else None
    sqrt_d = np.abs(oh.forward(psi, q, t, geo, s)) * rng.uniform(0.8, 1.2, (K, 4, n, n))
    sqrt_dref = np.abs(oh.reference_field(q, geo)) * 1.1
    return geo, np.ones_like(psi), q, t, s, sqrt_d, sqrt_dref


def _worker(rank, world, port, out, probe_shifts):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    geo, psi, q, t, s, sqrt_d, sqrt_dref = _problem(probe_shifts)
    k0, nk = shard(psi.shape[0], world, rank)
    geo_r = oh.Geometry(geo.wavelength, geo.pixel, geo.Z, geo.z, geo.n, geo.P,
                        w_ref=geo.w_ref if k0 == 0 else 0.0)
    F, gp, gq = oh.gradients(psi[k0:k0 + nk], q, t[k0:k0 + nk], sqrt_d[k0:k0 + nk], sqrt_dref,
                             geo_r, None if s is None else s[k0:k0 + nk])
    gq_t = torch.from_numpy(gq)
    F_all, gq_all = allreduce_loss_and_grad_q(F, gq_t)
    parts = [None] * world
    dist.all_gather_object(parts, (k0, nk, gp))
    if rank == 0:
        out.put((F_all, gq_all.numpy(), parts))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_covers_all_angles():
    for K in (1, 5, 60, 61):
        for world in (1, 2, 3, 8):
            got = [shard(K, world, r) for r in range(world)]
            assert got[0][0] == 0 and sum(nk for _, nk in got) == K
            assert all(got[i][0] + got[i][1] == got[i + 1][0] for i in range(world - 1))


@pytest.mark.parametrize("probe_shifts", [False, True])
def test_two_rank_shared_probe_gradient_equals_full(probe_shifts):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, probe_shifts)) for r in range(2)]
    for p in procs:
        p.start()
    F_all, gq_all, parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    geo, psi, qq, t, s, sqrt_d, sqrt_dref = _problem(probe_shifts)
    F, gp, gq = oh.gradients(psi, qq, t, sqrt_d, sqrt_dref, geo, s)
    assert F_all == pytest.approx(F, rel=1e-12)
    np.testing.assert_allclose(gq_all, gq, atol=1e-12 * np.abs(gq).max())
    for k0, nk, g in parts:
        np.testing.assert_allclose(g, gp[k0:k0 + nk], atol=1e-12 * np.abs(gp).max())


class _OracleHolo:
    """The library's evaluation calls, computed by the FP64 oracle on CPU tensors, so the
    GPU driver's sharded logic runs on gloo ranks without a GPU.  Covers the angles
    [k0g, k0g + K) of the problem; the reference term only if w_ref is set."""

    def __init__(self, geo, t, sqrt_d, sqrt_dref):
        self.geo, self.t, self.sqrt_d, self.sqrt_dref = geo, t, sqrt_d, sqrt_dref
        self.n_angles = self.chunk = t.shape[0]
        self.q = None

    def set_probe(self, q):
        self.q = q.numpy()

    def forward(self, psi, k0=0):
        nk = psi.shape[0]
        return oh.functional(psi.numpy(), self.q, self.t[k0:k0 + nk], self.sqrt_d[k0:k0 + nk],
                             self.sqrt_dref, self.geo)

    def gradient(self, psi, grad_psi, grad_q, k0=0, accumulate_q=False, loss_in=0.0):
        nk = psi.shape[0]
        F, gp, gq = oh.gradients(psi.numpy(), self.q, self.t[k0:k0 + nk],
                                 self.sqrt_d[k0:k0 + nk], self.sqrt_dref, self.geo)
        grad_psi.copy_(torch.from_numpy(gp))
        if accumulate_q:
            grad_q.add_(torch.from_numpy(gq))
            F += loss_in
        else:
            grad_q.copy_(torch.from_numpy(gq))
        return F, grad_psi, grad_q

    @staticmethod
    def dot(a, b):
        return float(np.real(np.vdot(a.numpy(), b.numpy())))

    def dy_dots(self, g, g_prev, eta):
        return self.dot(g, g), self.dot(g, eta), self.dot(g_prev, eta)

    @staticmethod
    def direction(eta, g, beta):
        eta.mul_(beta).sub_(g)

    @staticmethod
    def step(x, eta, gamma):
        x.add_(eta * gamma)


ITERS = 3


def _driver_worker(rank, world, port, out):
    import dataclasses

    import torch.distributed as dist
    from paper_2407_20304_gb300.cg import Reconstruction
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    geo, psi, q, t, _, sqrt_d, sqrt_dref = _problem(False)
    k0, nk = shard(psi.shape[0], world, rank)
    geo_r = dataclasses.replace(geo, w_ref=geo.w_ref if k0 == 0 else 0.0)
    h = _OracleHolo(geo_r, t[k0:k0 + nk], sqrt_d[k0:k0 + nk], sqrt_dref)
    r = Reconstruction(h, torch.from_numpy(psi[k0:k0 + nk].copy()), torch.from_numpy(q.copy()),
                       group=True)
    hist = r.run(ITERS)
    parts = [None] * world
    dist.all_gather_object(parts, (k0, nk, r.psi.numpy()))
    if rank == 0:
        out.put((hist, r.q.numpy(), parts))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_driver_follows_the_single_process_oracle_driver():
    """Reconstruction with a process group over 2 gloo ranks, the oracle standing in for
    each rank's evaluations: every loss, trial loss, grad_q and psi-block inner product is
    summed over the ranks, so the sharded run takes the single-process oracle driver's steps
    (same accepted step lengths, F history and iterates to rounding)."""
    from oracle import cg as ocg
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_driver_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    hist, q_fin, parts = q.get(timeout=600)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    geo, psi, qq, t, _, sqrt_d, sqrt_dref = _problem(False)
    ref = ocg.reconstruct(psi, qq, t, sqrt_d, sqrt_dref, geo, ITERS)
    assert hist["gamma_psi"] == ref["hist"]["gamma_psi"]
    assert hist["gamma_q"] == ref["hist"]["gamma_q"]
    np.testing.assert_allclose(hist["F"], ref["hist"]["F"], rtol=1e-10)
    np.testing.assert_allclose(hist["beta_psi"], ref["hist"]["beta_psi"], rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(q_fin, ref["q"], rtol=0, atol=1e-10 * np.abs(ref["q"]).max())
    for k0, nk, x in parts:
        np.testing.assert_allclose(x, ref["psi"][k0:k0 + nk], rtol=0,
                                   atol=1e-10 * np.abs(ref["psi"]).max())
    # the sharded run really moved both blocks
    assert any(g > 0 for g in hist["gamma_psi"]) and any(g > 0 for g in hist["gamma_q"])


def test_checkpoint_resume_is_bit_exact(tmp_path):
    """Driver state saved after 2 iterations and restored into a fresh driver continues
    exactly as an uninterrupted 4-iteration run (the oracle standing in for the library's
    evaluations, on CPU)."""
    from paper_2407_20304_gb300.cg import Reconstruction
    geo, psi, q, t, _, sqrt_d, sqrt_dref = _problem(False)

    def fresh(p0=psi, q0=q):
        h = _OracleHolo(geo, t, sqrt_d, sqrt_dref)
        return Reconstruction(h, torch.from_numpy(p0.copy()), torch.from_numpy(q0.copy()))

    full = fresh()
    full.run(4)
    part = fresh()
    part.run(2)
    path = tmp_path / "state.npz"
    part.save(path)
    res = fresh(np.zeros_like(psi), np.zeros_like(q))
    res.load(path)
    res.run(2)
    assert res.history == full.history
    assert torch.equal(res.psi, full.psi) and torch.equal(res.q, full.q)
    assert torch.equal(res.eta[0], full.eta[0]) and torch.equal(res.g[1], full.g[1])
    with pytest.raises(ValueError):
        Reconstruction(_OracleHolo(geo, t, sqrt_d, sqrt_dref), torch.from_numpy(psi.copy()),
                       torch.from_numpy(q.copy()), rule="polak-ribiere").load(path)


def test_driver_iteration_log(tmp_path):
    """The driver's JSONL log: one line per iteration, equal to its history, with the
    gradient norms and the relative error against a ground truth (oracle stand-in, CPU)."""
    import json
    from paper_2407_20304_gb300.cg import Reconstruction
    geo, psi, q, t, _, sqrt_d, sqrt_dref = _problem(False)
    path = tmp_path / "log.jsonl"
    truth = torch.from_numpy((0.9 + 0.05j) * np.ones_like(psi))
    r = Reconstruction(_OracleHolo(geo, t, sqrt_d, sqrt_dref), torch.from_numpy(psi.copy()),
                       torch.from_numpy(q.copy()), log_path=str(path), truth=truth)
    r.run(3)
    recs = [json.loads(line) for line in open(path)]
    assert [x["iter"] for x in recs] == [1, 2, 3]
    assert [x["F"] for x in recs] == r.history["F"][1:]
    assert [x["gamma_psi"] for x in recs] == r.history["gamma_psi"]
    assert [x["beta_q"] for x in recs] == r.history["beta_q"]
    assert all(x["gnorm_psi"] > 0 and x["gnorm_q"] > 0 for x in recs)
    d = r.psi.numpy().astype(np.complex128) - truth.numpy().astype(np.complex128)
    ref = np.linalg.norm(d) / np.linalg.norm(truth.numpy().astype(np.complex128))
    assert abs(recs[-1]["rel_err_psi"] - ref) <= 1e-9 * ref
