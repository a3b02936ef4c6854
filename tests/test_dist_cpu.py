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
