"""Multi-GPU layouts of the angle dimension (one process per GPU, torch.distributed).

* Independent chunks (the paper's production mode, Sec. 4): each rank reconstructs its own
  angle chunk with its own probe; nothing is exchanged.  `shard` gives the chunk.
* Shared probe: the angles of one problem are split over ranks; grad_psi_k stays on the
  rank that owns angle k, while F2 and grad_q are sums over all planes (Eq. min1 and the
  probe gradient after Eq. gradpsi), so each rank evaluates its planes and the partial loss
  and grad_q are summed with one all-reduce.  The reference-image term belongs to the rank
  that owns angle 0 (the library adds it when k0 == 0).
"""


def shard(n_angles, world, rank):
    """Contiguous angle range [k0, k0 + nk) of `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_angles, world)
    k0 = rank * base + min(rank, extra)
    return k0, base + (1 if rank < extra else 0)


def allreduce_loss_and_grad_q(loss, grad_q, group=None):
    """Sum the partial F2 (float) and grad_q (tensor, in place) over the ranks of `group`."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([loss], dtype=torch.float64, device=grad_q.device)
    dist.all_reduce(t, group=group)
    dist.all_reduce(grad_q, group=group)
    return float(t.item()), grad_q
