"""Joint psi / q reconstruction by nonlinear conjugate gradients (Sec. 2, Eq. DaiYuan2, and
the Fletcher-Reeves / Polak-Ribiere-Polyak formulas the paper names beside it).

The driver runs on the host and issues only library calls: gradients (passes A-D), trial
functionals for the line search (passes A-B), FP64 inner products for the Dai-Yuan
coefficient, and the vector updates.  Reading of the paper's unspecified line search (the
same reading as the FP64 oracle's driver): psi and q keep their own Dai-Yuan directions;
after one shared gradient the psi step is found by halving a trial step until F decreases,
then the q step the same way from the updated psi; a block whose trials never decrease F
keeps step 0, so F never increases; a non-positive DY denominator restarts the block with
-g; each block's next trial step is twice its last accepted one.  Options: the direction
rule ('dai-yuan', 'fletcher-reeves', 'polak-ribiere'; the latter two restart with -g when beta
is undefined or the new direction is not a descent direction) and the line search
('backtracking' as above, or 'armijo': the first halving with F <= F0 + 1e-4 gamma
Re <g, eta>, the q block using the gradient of the last evaluation).  The FP64 oracle driver
(oracle/cg.py) takes the same steps.  The initial probe of the paper (the reference image
propagated back to plane 0) is Holo.initial_probe.

Angles are processed in chunks of holo.chunk (the paper's independent angle chunks,
Sec. 4); the loss and grad_q are summed over chunks with the library's accumulate flag.

Shared probe over several processes (`group`, a torch.distributed process group, or the
default group when `group=True`): each rank holds its own slice of the angles (psi and its
context cover only those angles) and one copy of q.  F2 and grad_q are sums over all planes
(Eq. min1 and the probe gradient after Eq. gradpsi), so every gradient and every line-search
trial loss is summed over the ranks by an all-reduce, as are the psi block's inner products
(sums over the angles); grad_q is then the same on every rank, so the q block's products
need no exchange.  Every rank takes the same steps.  The reference-image term must be
counted once: only the rank that owns angle 0 creates its context with w_ref != 0.
"""

import json

import numpy as np
import torch


class Reconstruction:
    """State of a DY-CG reconstruction of psi [n_angles][n][n] and q [P][P] (CUDA, complex64)."""

    RULES = ("dai-yuan", "fletcher-reeves", "polak-ribiere")
    SEARCHES = ("backtracking", "armijo")
    ARMIJO_C = 1e-4

    def __init__(self, holo, psi, q, gamma0=1.0, max_halvings=20, update_q=True,
                 rule="dai-yuan", line_search="backtracking", group=None, log_path=None,
                 truth=None):
        """log_path: append one JSON line per iteration (iter, F, both steps and betas, the
        gradient norms, and with `truth` (psi's ground truth, laid out as psi) the relative
        error ||psi - truth|| / ||truth||); with a process group rank 0 writes it."""
        if rule not in self.RULES or line_search not in self.SEARCHES:
            raise ValueError(f"rule in {self.RULES}, line_search in {self.SEARCHES}")
        self.group = group
        self.h = holo
        self.psi = psi
        self.q = q
        self.gamma0 = gamma0
        self.max_halvings = max_halvings
        self.update_q = update_q
        self.rule = rule
        self.line_search = line_search
        self.trial = [gamma0, gamma0]
        self.g = None
        self.eta = None
        self.gg = [None, None]       # ||g||^2 of each block's current gradient
        self.slope = [None, None]    # Re <g, eta> of each block's current direction
        self.F = None
        self.history = {"F": [], "gamma_psi": [], "gamma_q": [], "beta_psi": [], "beta_q": [],
                        "F_after_psi": []}
        self.log_path = log_path
        self.truth = truth
        self._truth_sq = None

    # ------------------------------------------------------------------ reductions over ranks
    def _allreduce(self, vals):
        """Sum a list of floats over the ranks (FP64); unchanged without a group."""
        if self.group is None:
            return list(vals)
        import torch.distributed as dist
        grp = None if self.group is True else self.group
        t = torch.tensor(list(vals), dtype=torch.float64, device=self.psi.device)
        dist.all_reduce(t, group=grp)
        return t.tolist()

    def _allreduce_tensor(self, x):
        if self.group is not None:
            import torch.distributed as dist
            dist.all_reduce(x, group=None if self.group is True else self.group)
        return x

    def _dots(self, b, *pairs):
        """Re <a, c> for each pair; summed over the ranks for the psi block (b = 0)."""
        vals = [self.h.dot(a, c) for a, c in pairs]
        return self._allreduce(vals) if b == 0 else vals

    # ------------------------------------------------------------------ evaluations
    def _chunks(self):
        K, c = self.h.n_angles, self.h.chunk
        return [(k0, min(c, K - k0)) for k0 in range(0, K, c)]

    def functional(self, psi, q=None):
        """F2 at (psi, q); q = None keeps the probe last set (its propagations are reused)."""
        if q is not None:
            self.h.set_probe(q)
        F = sum(self.h.forward(psi[k0:k0 + nk], k0=k0) for k0, nk in self._chunks())
        return self._allreduce([F])[0]

    def gradient(self, psi, q, gpsi, gq):
        self.h.set_probe(q)
        loss = 0.0
        for i, (k0, nk) in enumerate(self._chunks()):
            loss, _, _ = self.h.gradient(psi[k0:k0 + nk], grad_psi=gpsi[k0:k0 + nk], grad_q=gq,
                                         k0=k0, accumulate_q=i > 0, loss_in=loss)
        self._allreduce_tensor(gq)
        return self._allreduce([loss])[0]

    # ------------------------------------------------------------------ iteration
    def _backtrack(self, f, x, eta, gamma, F0, scratch, slope):
        armijo = self.line_search == "armijo"
        if armijo and not slope < 0.0:
            return 0.0, F0
        for _ in range(self.max_halvings + 1):
            scratch.copy_(x)
            self.h.step(scratch, eta, gamma)
            Fx = f(scratch)
            if (Fx <= F0 + self.ARMIJO_C * gamma * slope) if armijo else (Fx < F0):
                x.copy_(scratch)
                return gamma, Fx
            gamma *= 0.5
        return 0.0, F0

    def _direction(self, b, g_new):
        """eta = -g_new + beta eta for the chosen rule; records ||g_new||^2 and the slope
        Re <g_new, eta_new> from the same inner products."""
        g_old, eta = self.g[b], self.eta[b]
        num, d_new, d_old = self.h.dy_dots(g_new, g_old, eta)
        if b == 0:
            num, d_new, d_old = self._allreduce([num, d_new, d_old])
        beta = None
        if self.rule == "dai-yuan":
            den = d_new - d_old
            beta = num / den if den > 0 else None
        else:
            oo = self.gg[b]
            if oo and oo > 0:
                if self.rule == "fletcher-reeves":
                    beta = num / oo
                else:
                    beta = (num - self._dots(b, (g_new, g_old))[0]) / oo
            if beta is not None and not (-num + beta * d_new) < 0.0:
                beta = None
        beta = 0.0 if beta is None else beta
        self.h.direction(eta, g_new, beta)
        self.gg[b] = num
        self.slope[b] = -num + beta * d_new
        return beta

    def run(self, iters):
        """Run `iters` iterations; returns the history of F and the accepted steps."""
        psi, q = self.psi, self.q
        if self.g is None:
            self.g = [torch.empty_like(psi), torch.empty_like(q)]
            self.F = self.gradient(psi, q, self.g[0], self.g[1])
            self.eta = [torch.zeros_like(psi), torch.zeros_like(q)]
            for b in range(2):
                self.h.direction(self.eta[b], self.g[b], 0.0)
                self.gg[b] = self._dots(b, (self.g[b], self.g[b]))[0]
                self.slope[b] = -self.gg[b]
            self.history["F"].append(self.F)
        scratch_psi, scratch_q = torch.empty_like(psi), torch.empty_like(q)
        g_new = [torch.empty_like(psi), torch.empty_like(q)]
        for _ in range(iters):
            self.h.set_probe(q)
            gam_psi, F = self._backtrack(lambda x: self.functional(x), psi, self.eta[0],
                                         self.trial[0], self.F, scratch_psi, self.slope[0])
            self.history["F_after_psi"].append(F)
            gam_q = 0.0
            if self.update_q:
                gam_q, F = self._backtrack(lambda x: self.functional(psi, x), q, self.eta[1],
                                           self.trial[1], F, scratch_q, self.slope[1])
            if gam_psi > 0:
                self.trial[0] = 2.0 * gam_psi
            if gam_q > 0:
                self.trial[1] = 2.0 * gam_q
            self.F = self.gradient(psi, q, g_new[0], g_new[1])
            betas = [self._direction(b, g_new[b]) for b in range(2)]
            self.g, g_new = g_new, self.g
            for key, val in (("F", self.F), ("gamma_psi", gam_psi), ("gamma_q", gam_q),
                             ("beta_psi", betas[0]), ("beta_q", betas[1])):
                self.history[key].append(val)
            if self.log_path is not None:
                self._log(gam_psi, gam_q, betas)
        return self.history

    def _log(self, gam_psi, gam_q, betas):
        rec = {"iter": len(self.history["F"]) - 1, "F": self.F, "gamma_psi": gam_psi,
               "gamma_q": gam_q, "beta_psi": betas[0], "beta_q": betas[1],
               "gnorm_psi": float(np.sqrt(max(self.gg[0], 0.0))),
               "gnorm_q": float(np.sqrt(max(self.gg[1], 0.0)))}
        if self.truth is not None:
            # ||psi - truth||^2 from FP64 inner products (no psi-sized temporary)
            if self._truth_sq is None:
                self._truth_sq = self._dots(0, (self.truth, self.truth))[0]
            pp, pt = self._dots(0, (self.psi, self.psi), (self.psi, self.truth))
            rec["rel_err_psi"] = float(np.sqrt(max(pp - 2.0 * pt + self._truth_sq, 0.0) /
                                               self._truth_sq))
        rank = 0
        if self.group is not None:
            import torch.distributed as dist
            rank = dist.get_rank()
        if rank == 0:
            with open(self.log_path, "a") as f:
                f.write(json.dumps(rec) + "\n")

    # ------------------------------------------------------------------ checkpoint / resume
    def save(self, path):
        """Write the driver state to an .npz file: psi, q, both blocks' gradients and
        directions, the next trial steps, ||g||^2 and the slopes of both blocks, F, and the
        history.  With a process group each rank saves its own psi slice (its own path)."""
        if self.g is None:
            raise RuntimeError("no state before the first gradient (run at least 0 iterations)")
        arrs = {"psi": self.psi, "q": self.q, "g_psi": self.g[0], "g_q": self.g[1],
                "eta_psi": self.eta[0], "eta_q": self.eta[1]}
        scal = np.array(self.trial + self.gg + self.slope + [self.F], np.float64)
        meta = json.dumps({"history": self.history, "rule": self.rule,
                           "line_search": self.line_search, "update_q": self.update_q,
                           "max_halvings": self.max_halvings, "gamma0": self.gamma0})
        np.savez(path, scalars=scal, meta=np.array(meta),
                 **{k: v.detach().cpu().numpy() for k, v in arrs.items()})

    def load(self, path):
        """Restore a state written by `save` into this driver: psi and q are overwritten in
        place (same shapes), the other tensors are allocated on psi's device.  The next `run`
        continues exactly where the saved one stopped."""
        with np.load(path) as f:
            meta = json.loads(str(f["meta"]))
            for k in ("rule", "line_search", "update_q", "max_halvings"):
                if meta[k] != getattr(self, k):
                    raise ValueError(f"checkpoint has {k}={meta[k]!r}, driver {getattr(self, k)!r}")
            arr = {k: torch.from_numpy(f[k]) for k in
                   ("psi", "q", "g_psi", "g_q", "eta_psi", "eta_q")}
            scal = f["scalars"].tolist()
        if arr["psi"].shape != self.psi.shape or arr["q"].shape != self.q.shape:
            raise ValueError("checkpoint shapes differ from this driver's psi / q")
        self.psi.copy_(arr["psi"])
        self.q.copy_(arr["q"])
        dev = self.psi.device
        self.g = [arr["g_psi"].to(dev), arr["g_q"].to(dev)]
        self.eta = [arr["eta_psi"].to(dev), arr["eta_q"].to(dev)]
        self.trial, self.gg, self.slope = scal[0:2], scal[2:4], scal[4:6]
        self.F = scal[6]
        self.gamma0 = meta["gamma0"]
        self.history = meta["history"]
