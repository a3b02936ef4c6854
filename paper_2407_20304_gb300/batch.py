"""Many independent reconstructions of uneven sizes evaluated by one CUDA-graph launch.

Two ways of issuing a batch evaluation are kept side by side:
* the persistent form (`prepare_persistent`, `capture_persistent`): the library's batch
  object (holo_batch_*) runs passes A-D of every round of chunks of all problems as persistent
  launches that walk device work lists of (problem, item) entries, one launch per pass and
  line length, captured once into a CUDA graph; `autotune_persistent` picks, per line length,
  the row passes' resident blocks per SM and pass B's TMA staging (coordinate descent, each
  candidate timed by graph replays);
* the per-problem form below: each problem's own launches, as a loop on one stream or
  captured into a graph whose branches run problems concurrently.
Both give every problem exactly the results of its own calls with the same schedule.


Each instance is its own problem (geometry, angles, distances, data, psi, q) with its own
library context; one evaluation of an instance is the probe propagation and the gradient
of F2 over all its angles (in chunks of the context's chunk size, the chunks summing
grad_q and the loss on the device).  `HoloBatch` issues the evaluations of all instances
either as a plain loop of launches on one stream, or captured once into a CUDA graph whose
branches run independent instances concurrently; replaying the graph evaluates the whole
batch with one launch from the host.

The schedule (how many concurrent branches, which instances on which branch) is chosen by
`autotune`: it measures each instance's evaluation time alone, balances the branches
longest-first for each candidate branch count, times one replay of each candidate graph,
and keeps the fastest.  Results do not depend on the schedule (every kernel is
deterministic and instances share no buffers).
"""

import ctypes
import time

import torch

from . import _lib


class Instance:
    """One reconstruction problem bound to a `Holo` context."""

    def __init__(self, holo, psi, q):
        self.h = holo
        self.psi = psi
        self.q = q
        self.grad_psi = torch.empty_like(psi)
        self.grad_q = torch.empty_like(q)

    def chunks(self):
        K, c = self.h.n_angles, self.h.chunk
        return [(k0, min(c, K - k0)) for k0 in range(0, K, c)]

    def issue(self):
        """Issue one evaluation on the context's stream (no host synchronisation): the chunks'
        probe-gradient sources are summed and propagated once (deferred grad_q)."""
        self.h.set_probe(self.q)
        for i, (k0, nk) in enumerate(self.chunks()):
            self.h.gradient(self.psi[k0:k0 + nk], grad_psi=self.grad_psi[k0:k0 + nk], k0=k0,
                            want_loss=False, accumulate_q=i > 0, defer_q=True)
        self.h.finish_q(self.grad_q)

    @property
    def planes(self):
        return self.h.n_angles * self.h.n_dist


class HoloBatch:
    def __init__(self, instances):
        self.inst = list(instances)
        self.main = torch.cuda.Stream()
        self.side = []
        self.graph = None
        self.schedule = None
        self.tuning = {}
        self._pbs = []           # holo_batch handles of the persistent form
        self.layout = None
        self.pgraph = None
        self.ptuning = {}

    @property
    def planes(self):
        return sum(i.planes for i in self.inst)

    # ------------------------------------------------------------------ loop
    def run_loop(self):
        """The per-instance launch loop on one stream."""
        for it in self.inst:
            it.h.set_stream(self.main)
            it.issue()

    def losses(self):
        return [it.h.read_loss() for it in self.inst]

    # ------------------------------------------------------------------ graph
    def _streams(self, nb):
        while len(self.side) < nb:
            self.side.append(torch.cuda.Stream())
        return self.side[:nb]

    def balanced(self, branches, cost):
        """Longest-processing-time-first assignment of instances to `branches` branches."""
        order = sorted(range(len(self.inst)), key=lambda i: -cost[i])
        load = [0.0] * branches
        groups = [[] for _ in range(branches)]
        for i in order:
            b = min(range(branches), key=lambda x: load[x])
            groups[b].append(i)
            load[b] += cost[i]
        return [g for g in groups if g]

    def capture(self, schedule):
        """Capture one evaluation of every instance, branch b of `schedule` on its own stream."""
        streams = self._streams(len(schedule))
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.main):
            cur = torch.cuda.current_stream()
            for s, members in zip(streams, schedule):
                s.wait_stream(cur)
                for i in members:
                    self.inst[i].h.set_stream(s)
                    self.inst[i].issue()
            for s in streams:
                cur.wait_stream(s)
        self.graph = g
        self.schedule = schedule
        return g

    def replay(self):
        """Launch the captured graph on the batch's stream."""
        with torch.cuda.stream(self.main):
            self.graph.replay()

    # ------------------------------------------------------------------ timing / tuning
    def _time(self, fn, reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.main)
        for _ in range(reps):
            fn()
        e1.record(self.main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def instance_costs(self):
        """Device time (ms) of one evaluation of each instance alone."""
        costs = []
        for it in self.inst:
            it.h.set_stream(self.main)
            it.issue()                      # warm-up
            costs.append(self._time(it.issue, 1))
        return costs

    def time_loop(self, reps=2):
        self.run_loop()
        return self._time(self.run_loop, reps)

    def autotune(self, candidates=(1, 2, 4, 8), reps=2):
        """Pick the branch count whose captured graph evaluates the batch fastest."""
        cost = self.instance_costs()
        best = None
        for nb in candidates:
            nb = min(nb, len(self.inst))
            sched = self.balanced(nb, cost)
            t0 = time.perf_counter()
            self.capture(sched)
            cap_s = time.perf_counter() - t0
            self.replay()
            ms = self._time(self.replay, reps)
            self.tuning[nb] = {"ms": ms, "capture_s": cap_s}
            if best is None or ms < best[0]:
                best = (ms, sched)
        self.capture(best[1])
        return best[0], best[1], cost

    # ------------------------------------------------------------------ persistent form
    def _check(self, st, where):
        if st != 0:
            raise _lib.HoloError(st, where, _lib.load().holo_last_error(self.inst[0].h.ctx).decode())

    def _groups(self, layout):
        """Instance indices per library batch: all in one ('one'), one batch per line length
        ('per_length'), or two per line length with the problems dealt alternately
        ('per_length_x2'); every batch but 'one' is issued on its own graph branch."""
        if layout == "one":
            return [list(range(len(self.inst)))]
        by = {}
        for i, it in enumerate(self.inst):
            by.setdefault(it.h.P, []).append(i)
        groups = [by[P] for P in sorted(by, reverse=True)]
        if layout == "per_length_x2":
            groups = [half for g in groups for half in (g[0::2], g[1::2]) if half]
        return groups

    def prepare_persistent(self, layout="one"):
        """Build the library's batch(es) over the instances (holo_batch_*), register their
        buffers and build the work lists (this sets pass_b_split = 0 on every context, so the
        per-problem loop gives the same results).  layout: 'one' batch for all, 'per_length'
        (one batch per line length) or 'per_length_x2' (two per line length), the batches of the
        last two on concurrent graph branches."""
        lib = _lib.load()
        self.close()
        self._pbs = []
        for members in self._groups(layout):
            arr = (ctypes.c_void_p * len(members))(*[self.inst[i].h.ctx.value for i in members])
            out = ctypes.c_void_p()
            self._check(lib.holo_batch_create(arr, len(members), ctypes.byref(out)),
                        "holo_batch_create")
            for slot, i in enumerate(members):
                it = self.inst[i]
                self._check(lib.holo_batch_set_problem(
                    out, slot, ctypes.c_void_p(it.psi.data_ptr()), ctypes.c_void_p(it.q.data_ptr()),
                    ctypes.c_void_p(it.grad_psi.data_ptr()), ctypes.c_void_p(it.grad_q.data_ptr())),
                    "holo_batch_set_problem")
            self._check(lib.holo_batch_prepare(out), "holo_batch_prepare")
            self._pbs.append(out)
        self.layout = layout

    def issue_persistent(self):
        """Issue one persistent-form evaluation of the whole batch: each library batch on its
        own branch stream, joined back into the current stream."""
        lib = _lib.load()
        cur = torch.cuda.current_stream()
        if len(self._pbs) == 1:
            self._check(lib.holo_batch_gradient(self._pbs[0], ctypes.c_void_p(cur.cuda_stream)),
                        "holo_batch_gradient")
            return
        streams = self._streams(len(self._pbs))
        for s, pb in zip(streams, self._pbs):
            s.wait_stream(cur)
            self._check(lib.holo_batch_gradient(pb, ctypes.c_void_p(s.cuda_stream)),
                        "holo_batch_gradient")
        for s in streams:
            cur.wait_stream(s)

    def capture_persistent(self):
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.main):
            self.issue_persistent()
        self.pgraph = g
        return g

    def replay_persistent(self):
        with torch.cuda.stream(self.main):
            self.pgraph.replay()

    def line_lengths(self):
        return sorted({it.h.P for it in self.inst}, reverse=True)

    def autotune_persistent(self, candidates=((0, -1), (2, -1), (0, 0), (2, 0)),
                            layouts=("one", "per_length", "per_length_x2"), reps=2):
        """The layout, then per line length the (row blocks per SM, pass-B stage) schedule,
        whose captured persistent graph evaluates the whole batch fastest: coordinate descent
        from the first candidate (layouts first, then line lengths in decreasing order), every
        trial timed by graph replays.  Returns (ms, {P: schedule}); self.layout holds the
        layout."""
        chosen = {P: candidates[0] for P in self.line_lengths()}

        def apply(sched, layout):
            for it in self.inst:
                rb, stage = sched[it.h.P]
                it.h.set_schedule(rb, stage, 0)
            self.prepare_persistent(layout)
            self.capture_persistent()
            self.replay_persistent()
            return self._time(self.replay_persistent, reps)

        best, best_layout = None, layouts[0]
        self.ptuning = {}
        for layout in layouts:
            ms = apply(chosen, layout)
            self.ptuning[f"layout {layout}"] = ms
            if best is None or ms < best:
                best, best_layout = ms, layout
        for P in self.line_lengths():
            for cand in candidates[1:]:
                trial = dict(chosen)
                trial[P] = cand
                ms = apply(trial, best_layout)
                self.ptuning[f"{best_layout} P={P} {cand}"] = ms
                if ms < best:
                    best, chosen = ms, trial
        apply(chosen, best_layout)
        return best, chosen

    def close(self):
        for pb in getattr(self, "_pbs", []) or []:
            _lib.load().holo_batch_destroy(pb)
        self._pbs = []
