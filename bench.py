#!/usr/bin/env python
"""Throughput of the holography gradient: plane-gradient evaluations per second.

One step is one pass of the whole hot path over one chunk of angles: probe propagation
(p_j = D_{omega_j} q, C D_{zeta_0} q), the fused forward / residual / adjoint passes
that give F2, grad_psi and grad_q (Eq. min1, Eq. gradpsi), the FP64 reductions, and the
Dai-Yuan conjugate-gradient update of psi and q (Eq. DaiYuan2: three FP64 inner
products, the direction update and the step x += gamma eta for each block).  A
plane-gradient evaluation is one (angle, distance) plane; a step over a chunk of K
angles and J distances is K*J of them.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one process per GPU (torchrun); each rank reconstructs its own angle chunk
(the paper's independent 150-angle chunks, Sec. 4), so per-GPU work is fixed (weak
scaling) and there is no data-path collective.  `--impl reference` times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import holo_synth as hs  # noqa: E402

METRIC = "plane-gradient evals/s at 2048^2 x 4 dist"
UNIT = "plane-grads/s"
KERNEL_SOURCES = ("paper_2407_20304_gb300/csrc/holo_kernels.cuh",
                  "paper_2407_20304_gb300/csrc/holo_fft.cuh")
FP32_LANES_PER_SM = 128
SMS = 152
MAX_SM_GHZ = 2.07


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default="large",
                    choices=("large", "autograd", "medium", "batch", "recon", "hier"))
    ap.add_argument("--recon-iters", type=int, default=200,
                    help="CG iterations of --workload recon (convergence run)")
    ap.add_argument("--functional", choices=("amplitude", "intensity"), default="amplitude",
                    help="F2 of Eq. min1 (amplitudes, the default) or F1 of Eq. min2 "
                         "(intensities); the unfused and oracle legs are F2 only")
    ap.add_argument("--probe-shifts", action="store_true",
                    help="probe shifts s_kj ~ U(-2, 2) px per axis and plane (Eq. min1), run by "
                         "the full-grid shift form of the passes; no unfused or oracle legs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--chunk", type=int, default=0,
                    help="angles per GPU (default: the workload's chunk); small values make "
                         "profiling captures small")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, n, planes):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the kernel
    sources are unchanged since it was taken and the launch has the captured size (else
    None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(kernel)
    if not e or e.get("kernel_hash") != kernel_hash():
        return None
    if e.get("n") != n or e.get("full_launch_planes") != planes:
        return None
    return e.get("bytes_per_launch_full")


# ---------------------------------------------------------------- geometry helpers

def derived(z, Z):
    z = np.asarray(z, float)
    mt = z / z[0]
    zeta = z * (Z - z) / Z
    return mt, zeta


def boxes(n, P, mt, shifts):
    """Box sizes (bys, bxs) per plane, as the library computes them (support of R0)."""
    def ax(m, t):
        a = P // 2 + (t - n // 2 - 1.0) / m
        b = P // 2 + (t + n // 2) / m
        s, e = int(np.floor(a)) - 1, int(np.ceil(b)) + 2
        return max(min(e, P) - max(s, 0), 0)
    K, J = shifts.shape[:2]
    return [[(ax(mt[j], shifts[k, j, 0]), ax(mt[j], shifts[k, j, 1])) for j in range(J)]
            for k in range(K)]


def algorithmic_costs(n, P, box, ref=True):
    """Per-pass algorithmic HBM bytes and FP32 flops over the chunk (sum over planes).

    FFT flops use the 5 N log2 N convention for a complex FFT of length N; bytes count
    each input read and output written once (complex64 = 8 B, amplitudes 4 B).  Per plane
    with box sy x sx: pass A reads psi (its n x n footprint) and p_j on the box and writes
    w (box) and Y (sy x n); pass B reads Y and the data and writes V (sy x n), and once per
    launch reads b = C D_{zeta_0} q and r_ref and writes T (n x n each); pass C reads V,
    p_j and w on the box and writes conj(w) v (box) and h (sy x n); pass D reads h and
    writes grad_psi once per angle."""
    fft = 5.0 * P * np.log2(P)
    K, J = len(box), len(box[0])
    out = {k: {"bytes": 0.0, "flops": 0.0} for k in ("pass_a", "pass_b", "pass_c", "pass_d")}
    for k in range(K):
        for j in range(J):
            sy, sx = box[k][j]
            out["pass_a"]["bytes"] += 8 * n * n + 16 * sy * sx + 8 * sy * n
            out["pass_a"]["flops"] += sy * (2 * fft + 6 * P) + 30 * sy * sx
            out["pass_b"]["bytes"] += 16 * sy * n + 4 * n * n
            out["pass_b"]["flops"] += n * (4 * fft + 12 * P) + 20 * n * n
            out["pass_c"]["bytes"] += 16 * sy * n + 24 * sy * sx
            out["pass_c"]["flops"] += sy * (2 * fft + 6 * P) + 60 * sy * sx
            out["pass_d"]["bytes"] += 8 * sy * n
            out["pass_d"]["flops"] += 8 * n * n
        out["pass_d"]["bytes"] += 8 * n * n
    out["pass_b"]["bytes"] += (24 if ref else 16) * n * n
    return out


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workload

def workload_inputs(w, rank):
    """psi_true, q_true, shifts of the rank's chunk (seeded by the workload and rank)."""
    rng = hs.rng_for(w.seed, rank)
    angles = range(rank * w.chunk, rank * w.chunk + w.chunk)
    psi_true = hs.object_stack(w, angles, rng).astype(np.complex64)
    q_true = hs.striped_probe(w.P, w.probe_sigma, rng).astype(np.complex64)
    shifts = hs.sample_shifts(w.chunk, w.n_dist, rng).astype(np.float32)
    q0 = hs.perturbed_probe(q_true, rng).astype(np.complex64)
    return psi_true, q_true, shifts, q0


def run_ours(args, w, rank, world, local_rank):
    import torch
    from paper_2407_20304_gb300 import Holo
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    g = hs.WORKLOAD_GEOMETRY
    n, P, K, J = w.n, w.P, w.chunk, w.n_dist
    psi_true, q_true, shifts, q0 = workload_inputs(w, rank)
    h = Holo(n, K, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], pad=P, chunk=K)
    if args.probe_shifts:
        srng = hs.rng_for(w.seed + 77, rank)
        h.set_probe_shifts(srng.uniform(-2.0, 2.0, (K, J, 2)).astype(np.float32))
        args.no_unfused = args.no_cpu = True
    h.set_shifts(shifts)
    # synthetic data: |u|^2 of the true object and probe, Poisson noise at w.counts counts
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.seed + rank)
    psi_t = torch.from_numpy(psi_true).to(dev)
    qt = torch.from_numpy(q_true).to(dev)
    h.set_probe(qt)
    u = torch.empty((K, J, n, n), dtype=torch.complex64, device=dev)
    h.set_data(torch.ones((K, J, n, n), dtype=torch.float32, device=dev),
               torch.ones((n, n), dtype=torch.float32, device=dev))
    h.forward(psi_t, u_out=u)
    inten = u.abs().square_()
    del u
    c = w.counts / inten.mean()
    sqrt_d = torch.poisson(inten.mul_(c), generator=gen).div_(c).sqrt_()
    del inten
    _, zeta = derived(g["z"][:J], g["Z"])
    lo = P // 2 - n // 2
    bref = h.propagate(qt, zeta[0])[lo:lo + n, lo:lo + n]
    iref = bref.abs().square()
    cr = w.counts / iref.mean()
    sqrt_dref = torch.poisson(iref * cr, generator=gen).div_(cr).sqrt_().contiguous()
    f1 = args.functional == "intensity"
    if f1:
        # F1 reads intensities: the same Poisson data, squared back
        h.set_functional("intensity")
        sqrt_d.square_()
        sqrt_dref.square_()
        args.no_unfused = args.no_cpu = True
    h.set_data(sqrt_d, sqrt_dref)
    del psi_t, qt

    psi = torch.ones((K, n, n), dtype=torch.complex64, device=dev)
    q = torch.from_numpy(q0).to(dev)
    gpsi = [torch.empty_like(psi), torch.empty_like(psi)]
    gq = [torch.empty_like(q), torch.empty_like(q)]
    eta_psi, eta_q = torch.zeros_like(psi), torch.zeros_like(q)
    state = {"cur": 0, "first": True, "gam": None}

    def step():
        cur = state["cur"]
        h.set_probe(q)
        loss, gp, gqc = h.gradient(psi, grad_psi=gpsi[cur], grad_q=gq[cur])
        if state["gam"] is None:
            # fixed small steps (relative 1e-3 of each block) for the benchmark's updates
            state["gam"] = (1e-3 * (K * n * n) ** 0.5 / max(np.sqrt(h.dot(gp, gp)), 1e-30),
                            1e-3 * np.sqrt(h.dot(q, q)) / max(np.sqrt(h.dot(gqc, gqc)), 1e-30))
        for gcur, gprev, eta, x, gam in ((gp, gpsi[1 - cur], eta_psi, psi, state["gam"][0]),
                                         (gqc, gq[1 - cur], eta_q, q, state["gam"][1])):
            beta = 0.0
            if not state["first"]:
                num, d_new, d_old = h.dy_dots(gcur, gprev, eta)
                den = d_new - d_old
                beta = num / den if den > 0 else 0.0
            h.direction_step(x, eta, gcur, beta, gam)
        state["first"] = False
        state["cur"] = 1 - cur
        return loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    planes = K * J * world
    # end to end through the host-buffer entry point, measured after the warm-up steps and
    # before the device-timed loop (host<->device copy rates of the box drop after long
    # sustained load, while device compute does not)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(h, args, w, psi, q, sqrt_d, dev, planes, dist)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[local_rank]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local_rank
    l0 = h.launch_count()
    h.set_timing(True)
    with ClockSampler(gpu_index) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            loss = step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = h.launch_count() - l0
    timing = h.get_timing()
    h.set_timing(False)
    if dist:
        t = torch.tensor([ms], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        ms = float(t.item())
        tdist.barrier()
    value = planes * args.steps / (ms / 1e3)

    # roofline of the dominant kernel
    mt, _ = derived(g["z"][:J], g["Z"])
    box = [[(P, P)] * J] * K if args.probe_shifts else boxes(n, P, mt, shifts)
    costs = algorithmic_costs(n, P, box)
    passes = [p for p in ("pass_a", "pass_b", "pass_c", "pass_d")]
    top = max(passes, key=lambda p: timing[p][0])
    top_ms = timing[top][0] / max(timing[top][1], 1)
    pk = peaks()
    gbs = costs[top]["bytes"] / (top_ms / 1e3) / 1e9
    tfl = costs[top]["flops"] / (top_ms / 1e3) / 1e12
    clocks = clk.summary()
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * MAX_SM_GHZ / 1e3
    hbm_frac, alu_frac = gbs / pk["hbm_gbs"], tfl / fp32_peak
    traffic = None if args.probe_shifts else recorded_traffic(top, n, K * J)
    if alu_frac >= hbm_frac:
        roof = {"bound": "alu", "achieved": round(tfl, 2), "peak": round(fp32_peak, 1),
                "unit": "TFLOP/s", "frac": round(alu_frac, 4), "traffic": traffic,
                "kernel": top, "hbm_gbs": round(gbs, 1), "hbm_frac": round(hbm_frac, 4),
                "peak_source": f"FP32: {SMS} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{MAX_SM_GHZ} GHz; HBM {pk['source']} {pk['hbm_gbs']} GB/s"}
    else:
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(hbm_frac, 4), "traffic": traffic, "kernel": top,
                "alu_tflops": round(tfl, 2), "alu_frac": round(alu_frac, 4),
                "peak_source": f"HBM {pk['source']}"}
    per_pass = {p: {"ms_per_step": round(timing[p][0] / args.steps, 3),
                    "launches_per_step": timing[p][1] / args.steps}
                for p in hs_timers()}

    unfused = None
    if not args.no_unfused:
        shifts_np = shifts.astype(np.float64)
        unfused = run_unfused_sample(w, torch.ones_like(psi), torch.from_numpy(q0).to(dev),
                                     shifts_np, sqrt_d, sqrt_dref)
    result = {
        "metric": METRIC + (" (F1 intensity functional)" if f1 else "")
                  + (" (probe shifts)" if args.probe_shifts else ""), "value": round(value, 1),
        "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{w.name}: psi {n}^2 (pad {P}), {K}-angle chunk x {J} distances "
                               f"per GPU, layered phantom, striped probe, Poisson {w.counts:g}",
                   "n": n, "pad": P, "angles_per_gpu": K, "n_dist": J,
                   "planes_per_step": planes, "reductions": "f64",
                   "l2": "inputs larger than L2 (psi chunk %.1f GB, data %.1f GB per GPU)"
                         % (K * n * n * 8 / 1e9, K * J * n * n * 4 / 1e9),
                   "functional": "F1 (Eq. min2, intensities)" if f1 else "F2 (Eq. min1, amplitudes)",
                   "probe_shifts": ("U(-2, 2) px per axis and plane, full-grid shift form"
                                    if args.probe_shifts else "none"),
                   "step": "set_probe + gradient (F, grad_psi, grad_q) + DY inner products + fused direction/step"},
        "roofline": roof, "clocks": clocks, "gpu_launches": launches, "per_pass": per_pass,
        "final_loss": loss,
    }
    if e2e:
        result["e2e"] = e2e
    if unfused:
        result["unfused_cufft"] = unfused
    return result, h


def hs_timers():
    from paper_2407_20304_gb300 import _lib
    return _lib.TIMERS


def run_e2e(h, args, w, psi, q, sqrt_d, dev, planes, dist):
    """Same metric through holo_gradient_host: inputs copied from pinned host memory and
    results read back inside the timed region, every step."""
    import torch
    K, J, n, P = w.chunk, w.n_dist, w.n, w.P
    pin = dict(pin_memory=True)
    psi_h = torch.empty((K, n, n), dtype=torch.complex64, **pin)
    psi_h.copy_(psi)
    d_h = torch.empty((K, J, n, n), dtype=torch.float32, **pin)
    d_h.copy_(sqrt_d)
    q_h = torch.empty((P, P), dtype=torch.complex64, **pin)
    q_h.copy_(q)
    gp_h = torch.empty((K, n, n), dtype=torch.complex64, **pin)
    gq_h = torch.empty((P, P), dtype=torch.complex64, **pin)
    a = [x.numpy() for x in (psi_h, d_h, q_h, gp_h, gq_h)]
    h.gradient_host(a[0], sqrt_d=a[1], q=a[2], grad_psi=a[3], grad_q=a[4])
    steps = max(3, min(args.steps, 10))
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        h.gradient_host(a[0], sqrt_d=a[1], q=a[2], grad_psi=a[3], grad_q=a[4])
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if dist:
        t = torch.tensor([dt], device=dev)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        dt = float(t.item())
    h2d = psi_h.numel() * 8 + d_h.numel() * 4 + q_h.numel() * 8
    d2h = gp_h.numel() * 8 + gq_h.numel() * 8 + 16
    return {"value": round(planes * steps / dt, 1), "unit": UNIT, "steps": steps,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "holo_gradient_host (psi, data, q host -> grad_psi, grad_q, loss host)"}


# ---------------------------------------------------------------- unfused comparison

class Unfused:
    """The same F2 and gradients in the plain unfused per-plane form: cuFFT 2D transforms
    (torch.fft) on the full P x P grid and separate elementwise kernels (resample by
    separable gathers, chirp products, crop, residual, zero embedding, adjoint resample by
    index_add_, G_j accumulation).  A timed comparison only; not part of the library."""

    def __init__(self, n, P, geom, shifts, sqrt_d, sqrt_dref, ext=1.0, w_ref=1.0, device="cuda"):
        import torch
        self.t = torch
        self.n, self.P, self.ext, self.w_ref = n, P, ext, w_ref
        z = np.asarray(geom["z"], float)
        Z, lam, dx = geom["Z"], geom["wavelength"], geom["pixel"]
        mt = z / z[0]
        self.mt = mt
        omega, zeta = (z - z[0]) / mt, z * (Z - z) / Z
        zhat = zeta / mt ** 2
        k = np.arange(P, dtype=float)
        k[k >= P // 2] -= P
        f2 = (k / (P * dx)) ** 2
        f2d = f2[:, None] + f2[None, :]

        def H(dist):
            return torch.from_numpy(np.exp(-1j * np.pi * lam * dist * f2d).astype(np.complex64)).to(device)
        self.Hz = [H(d) for d in zhat]
        self.Ho = [H(d) for d in omega]
        self.Hr = H(zeta[0])
        self.shifts = shifts
        self.sqrt_d = sqrt_d            # [K][J][n][n] torch cuda
        self.sqrt_dref = sqrt_dref
        self.dev = device
        self.J = len(z)

    def _taps(self, mtj, tj):
        t = self.t
        X = t.arange(self.P, device=self.dev, dtype=t.float64) - self.P // 2
        xi = mtj * X - tj + self.n // 2
        i0 = t.floor(xi)
        f = (xi - i0).float()
        i0 = i0.long()
        return i0, f

    def _axis(self, i0, f):
        """taps (index, weight*mask) for the two neighbours along one axis."""
        n = self.n
        out = []
        for di, w in ((0, 1 - f), (1, f)):
            idx = i0 + di
            m = (idx >= 0) & (idx < n)
            out.append((idx.clamp(0, n - 1), w * m.float()))
        return out

    def resample(self, psi, ky, kx):
        """ext + R0(psi - ext) on the P x P grid (separable bilinear)."""
        d = psi - self.ext
        rows = sum(w[:, None] * d.index_select(0, idx) for idx, w in ky)          # [P][n]
        full = sum(w[None, :] * rows.index_select(1, idx) for idx, w in kx)       # [P][P]
        return full + self.ext

    def resample_T(self, g, ky, kx):
        t = self.t
        n = self.n
        cols = t.zeros((self.P, n), dtype=g.dtype, device=self.dev)
        for idx, w in kx:
            cols.index_add_(1, idx, g * w[None, :])
        out = t.zeros((n, n), dtype=g.dtype, device=self.dev)
        for idx, w in ky:
            out.index_add_(0, idx, cols * w[:, None])
        return out

    def gradient(self, psi, q):
        t = self.t
        n, P, J = self.n, self.P, self.J
        lo = P // 2 - n // 2
        fft2, ifft2 = t.fft.fft2, t.fft.ifft2
        p = [q] + [ifft2(fft2(q) * self.Ho[j]) for j in range(1, J)]
        gpsi = t.zeros_like(psi)
        G = [t.zeros((P, P), dtype=t.complex64, device=self.dev) for _ in range(J)]
        loss = 0.0
        for k in range(psi.shape[0]):
            for j in range(J):
                ty, tx = float(self.shifts[k, j, 0]), float(self.shifts[k, j, 1])
                ky = self._axis(*self._taps(float(self.mt[j]), ty))
                kx = self._axis(*self._taps(float(self.mt[j]), tx))
                Rpsi = self.resample(psi[k], ky, kx)
                u = ifft2(fft2(p[j] * Rpsi) * self.Hz[j])[lo:lo + n, lo:lo + n]
                a = self.sqrt_d[k, j]
                mag = u.abs()
                loss += float(((mag - a) ** 2).sum(dtype=t.float64))
                r = u * t.where(mag > 0, 1 - a / mag, t.zeros_like(mag))
                e = t.zeros((P, P), dtype=t.complex64, device=self.dev)
                e[lo:lo + n, lo:lo + n] = r
                v = ifft2(fft2(e) * t.conj(self.Hz[j]))
                gpsi[k] += 2 * self.resample_T(t.conj(p[j]) * v, ky, kx)
                G[j] += t.conj(Rpsi) * v
        gq = sum(2 * ifft2(fft2(G[j]) * t.conj(self.Ho[j])) for j in range(J))
        if self.w_ref:
            b = ifft2(fft2(q) * self.Hr)[lo:lo + n, lo:lo + n]
            mag = b.abs()
            loss += self.w_ref * float(((mag - self.sqrt_dref) ** 2).sum(dtype=t.float64))
            rr = b * t.where(mag > 0, 1 - self.sqrt_dref / mag, t.zeros_like(mag))
            e = t.zeros((P, P), dtype=t.complex64, device=self.dev)
            e[lo:lo + n, lo:lo + n] = rr
            gq = gq + 2 * self.w_ref * ifft2(fft2(e) * t.conj(self.Hr))
        return loss, gpsi, gq


def run_unfused_sample(w, psi, q, shifts, sqrt_d, sqrt_dref, angles=4):
    """Plane-gradients/s of the unfused cuFFT form on `angles` angles of the workload."""
    import torch
    g = hs.WORKLOAD_GEOMETRY
    u = Unfused(w.n, w.P, g, shifts[:angles], sqrt_d[:angles], sqrt_dref)
    u.gradient(psi[:1], q)          # warm-up (plans, allocator)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    u.gradient(psi[:angles], q)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": round(angles * w.n_dist / (ms / 1e3), 1), "unit": UNIT,
            "sample": f"{angles} angles x {w.n_dist} distances, one gradient evaluation incl. "
                      f"probe propagation and grad_q",
            "impl": "torch.fft (cuFFT) 2D transforms on the P x P grid + separate elementwise "
                    "kernels, FP32"}


# ---------------------------------------------------------------- oracle (CPU)

_ORACLE_INPUTS = {}


def oracle_setup(w):
    """Inputs of the oracle samples: the first angle of the workload at the start point
    psi = 1, with data |u| of the true object made by the oracle itself (made once per
    workload and process)."""
    key = (w.name, w.n, w.P, w.n_dist, w.seed)
    if key not in _ORACLE_INPUTS:
        _ORACLE_INPUTS[key] = _oracle_inputs(w)
    return _ORACLE_INPUTS[key]


def _oracle_inputs(w):
    from oracle import holo as oh
    g = hs.WORKLOAD_GEOMETRY
    rng = hs.rng_for(w.seed, 0)
    psi_true = hs.object_stack(w, range(1), rng)
    q_true = hs.striped_probe(w.P, w.probe_sigma, rng)
    shifts = hs.sample_shifts(1, w.n_dist, rng).astype(np.float32).astype(np.float64)
    geo = oh.Geometry(g["wavelength"], g["pixel"], g["Z"], tuple(g["z"][:w.n_dist]), w.n, w.P)
    sqrt_d = np.abs(oh.forward(psi_true, q_true, shifts, geo))[0]
    return np.ones((w.n, w.n), np.complex128), q_true, shifts, sqrt_d, geo


def oracle_plane(inputs, j):
    from oracle import holo as oh
    psi0, q, shifts, sqrt_d, geo = inputs
    jj = j % geo.n_dist
    return oh.plane_gradient(psi0, q, shifts[0, jj], sqrt_d[jj], geo, jj)


def cpu_baseline(w, budget_s):
    """The CPU leg: the oracle as it stands, timed on the host cores for about `budget_s`
    seconds, and the FP32 error of the GPU path against it on one angle of the workload.
    Returns (baseline, error report)."""
    err = precision_report(w)
    inputs = oracle_setup(w)
    done, t_used = 0, 0.0
    while done < 1 or t_used < budget_s:
        t0 = time.perf_counter()
        oracle_plane(inputs, done)
        t_used += time.perf_counter() - t0
        done += 1
    return {"value": round(done / t_used, 4), "unit": UNIT, "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"{done} plane-gradient(s) of the {w.name} workload (n={w.n}, P={w.P}, "
                      f"first angle, distances cycled) by the FP64 oracle in {t_used:.1f} s; "
                      f"scipy.fft on all host cores"}, err


def precision_report(w):
    """Part of the CPU leg: relative L2 error of the FP32 GPU loss and gradients against the
    FP64 oracle on one angle (all distances, reference term included) of the workload at the
    start point psi = 1, q = the true probe: the oracle's own noiseless data, inputs rounded
    to the GPU's types and given to both sides.  Also returns the oracle's time for that
    evaluation."""
    import torch
    from oracle import holo as oh
    from paper_2407_20304_gb300 import Holo
    psi0, q, shifts, sqrt_d, geo = oracle_setup(w)
    q = q.astype(np.complex64).astype(np.complex128)
    sqrt_d = sqrt_d.astype(np.float32).astype(np.float64)
    sqrt_dref = np.abs(oh.reference_field(q, geo)).astype(np.float32).astype(np.float64)
    J, n, P = geo.n_dist, geo.n, geo.P
    t0 = time.perf_counter()
    F, gp_ref, gq_ref = oh.gradients(psi0[None], q, shifts, sqrt_d[None], sqrt_dref, geo)
    t_oracle = time.perf_counter() - t0
    g = hs.WORKLOAD_GEOMETRY
    h = Holo(n, 1, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], pad=P)
    dev = torch.device("cuda", torch.cuda.current_device())
    h.set_shifts(shifts.astype(np.float32))
    d_sd = torch.tensor(sqrt_d[None], dtype=torch.float32, device=dev)
    d_ref = torch.tensor(sqrt_dref, dtype=torch.float32, device=dev)
    h.set_data(d_sd, d_ref)
    h.set_probe(torch.tensor(q, dtype=torch.complex64, device=dev))
    loss, gp, gq = h.gradient(torch.tensor(psi0[None], dtype=torch.complex64, device=dev))
    torch.cuda.synchronize()
    h.close()

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    return {"loss": abs(loss - F) / abs(F), "grad_psi": rel(gp.cpu().numpy(), gp_ref[0]),
            "grad_q": rel(gq.cpu().numpy(), gq_ref), "oracle_s": round(t_oracle, 2),
            "sample": f"angle 0 x {J} distances of the {w.name} workload (n={n}, P={P}) with the "
                      "reference term, at psi = 1 and the true probe, oracle-made noiseless "
                      "data; relative L2 against the FP64 oracle (targets: loss 1e-5, "
                      "gradients 1e-4)"}


def run_reference(args, w):
    """The reference arm: the oracle timed as it stands, one plane-gradient per step."""
    inputs = oracle_setup(w)
    for s in range(args.warmup):
        oracle_plane(inputs, s)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle_plane(inputs, s)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = (f"{args.steps} plane-gradients of the {w.name} workload (n={w.n}, P={w.P}), one "
              f"per step, FP64 oracle with scipy.fft on all host cores")
    return {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"{w.name}: psi {w.n}^2 (pad {w.P}), {w.chunk}-angle chunk x "
                                   f"{w.n_dist} distances per GPU, layered phantom, striped probe, "
                                   f"Poisson {w.counts:g}",
                       "sample": "one plane-gradient of that workload per timed step"},
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- reconstruction (convergence)

def run_recon(args):
    """Joint psi / q DY-CG reconstructions (Sec. 2) on a 16-angle chunk of the medium workload
    (psi 512^2 on 1024^2, 4 distances, layered phantom, striped probe), from psi = 1 and the
    paper's initial probe (the reference image propagated back to plane 0), on noise-free and
    on Poisson (1e4 counts) data: F per iteration and the relative errors of psi and q against
    the synthetic truth, as in Fig. conv.  Wall-clock time of the whole driver (host-driven,
    line searches included)."""
    import torch
    from paper_2407_20304_gb300 import Holo
    from paper_2407_20304_gb300.cg import Reconstruction
    import __graft_entry__
    __graft_entry__.build()
    w = hs.workloads()["medium"]
    g = hs.WORKLOAD_GEOMETRY
    n, P, J, K = w.n, w.P, w.n_dist, 16
    rng = hs.rng_for(w.seed, 31)
    psi_true = torch.from_numpy(hs.object_stack(w, range(K), rng).astype(np.complex64)).cuda()
    q_true = torch.from_numpy(hs.striped_probe(P, w.probe_sigma, rng).astype(np.complex64)).cuda()
    shifts = hs.sample_shifts(K, J, rng).astype(np.float32)
    _, zeta = derived(g["z"][:J], g["Z"])
    lo = P // 2 - n // 2
    runs = {}
    for label, counts in (("noise-free", None), ("noisy", w.counts)):
        h = Holo(n, K, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], pad=P)
        h.set_shifts(shifts)
        h.set_data(torch.ones((K, J, n, n), dtype=torch.float32, device="cuda"),
                   torch.ones((n, n), dtype=torch.float32, device="cuda"))
        h.set_probe(q_true)
        u = torch.empty((K, J, n, n), dtype=torch.complex64, device="cuda")
        h.forward(psi_true, u_out=u)
        inten = u.abs().square()
        iref = h.propagate(q_true, zeta[0])[lo:lo + n, lo:lo + n].abs().square()
        if counts:
            gen = torch.Generator(device="cuda").manual_seed(w.seed + 77)
            c = counts / inten.mean()
            inten = torch.poisson(inten * c, generator=gen) / c
            cr = counts / iref.mean()
            iref = torch.poisson(iref * cr, generator=gen) / cr
        sqrt_d, sqrt_dref = inten.sqrt().contiguous(), iref.sqrt().contiguous()
        h.set_data(sqrt_d, sqrt_dref)
        q0 = h.initial_probe(sqrt_dref)
        psi = torch.ones((K, n, n), dtype=torch.complex64, device="cuda")
        rec = Reconstruction(h, psi, q0.clone())
        err = {"psi": [], "q": []}
        checkpoints = []
        t_run = 0.0
        done = 0
        step = 10
        while done < args.recon_iters:
            m = min(step, args.recon_iters - done)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rec.run(m)
            torch.cuda.synchronize()
            t_run += time.perf_counter() - t0
            done += m
            checkpoints.append(done)
            err["psi"].append(float((rec.psi - psi_true).norm() / psi_true.norm()))
            err["q"].append(float((rec.q - q_true).norm() / q_true.norm()))
        F = rec.history["F"]
        gaps = sum(1 for a, b in zip(rec.history["gamma_psi"], rec.history["gamma_q"]) if a == 0 or b == 0)
        runs[label] = {"iterations": done, "seconds": round(t_run, 3),
                       "iterations_per_s": round(done / t_run, 2),
                       "F_first": F[0], "F_last": F[-1],
                       "F_every_10": [F[i] for i in checkpoints],
                       "rel_err_psi_every_10": err["psi"], "rel_err_q_every_10": err["q"],
                       "monotone": all(b <= a for a, b in zip(F, F[1:])),
                       "iterations_with_a_zero_step": gaps}
        h.close()
    return {"metric": "CG iterations/s, joint psi/q reconstruction (16 angles, 512^2 on 1024^2, 4 dist)",
            "value": runs["noise-free"]["iterations_per_s"], "unit": "it/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "recon: medium workload chunk, psi0 = 1, q0 = reference image "
                                   "propagated back to plane 0, DY directions, backtracking",
                       "iterations": args.recon_iters},
            "runs": runs}


def run_hier(args):
    """Hierarchical reconstruction (Sec. 3) against a flat one with the same wall-clock budget
    on the recon problem (16 angles of the medium workload, noise-free data): levels bin 8, 4,
    2, 1 with 400, 200, 100, 50 iterations, then the unbinned driver alone for as long as the
    hierarchy took.  Reports F on the full grid and the psi error of both."""
    import torch
    from paper_2407_20304_gb300 import Holo
    from paper_2407_20304_gb300.cg import Reconstruction
    from paper_2407_20304_gb300.hierarchy import Hierarchy
    import __graft_entry__
    __graft_entry__.build()
    w = hs.workloads()["medium"]
    g = hs.WORKLOAD_GEOMETRY
    n, P, J, K = w.n, w.P, w.n_dist, 16
    rng = hs.rng_for(w.seed, 31)
    psi_true = torch.from_numpy(hs.object_stack(w, range(K), rng).astype(np.complex64)).cuda()
    q_true = torch.from_numpy(hs.striped_probe(P, w.probe_sigma, rng).astype(np.complex64)).cuda()
    shifts = hs.sample_shifts(K, J, rng).astype(np.float32)
    _, zeta = derived(g["z"][:J], g["Z"])
    lo = P // 2 - n // 2
    h = Holo(n, K, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], pad=P)
    h.set_shifts(shifts)
    h.set_data(torch.ones((K, J, n, n), dtype=torch.float32, device="cuda"),
               torch.ones((n, n), dtype=torch.float32, device="cuda"))
    h.set_probe(q_true)
    u = torch.empty((K, J, n, n), dtype=torch.complex64, device="cuda")
    h.forward(psi_true, u_out=u)
    sqrt_d = u.abs().contiguous()
    sqrt_dref = h.propagate(q_true, zeta[0])[lo:lo + n, lo:lo + n].abs().contiguous()
    del u
    h.set_data(sqrt_d, sqrt_dref)
    levels = ((8, 400), (4, 200), (2, 100), (1, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hier = Hierarchy(n, K, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], shifts, pad=P,
                     levels=levels)
    psi_h, q_h = hier.run(sqrt_d, sqrt_dref)
    torch.cuda.synchronize()
    t_hier = time.perf_counter() - t0
    h.set_probe(q_h)
    F_h = h.forward(psi_h)
    err_h = float((psi_h - psi_true).norm() / psi_true.norm())
    # flat: the unbinned driver for the same wall time
    q0 = h.initial_probe(sqrt_dref)
    rec = Reconstruction(h, torch.ones((K, n, n), dtype=torch.complex64, device="cuda"), q0.clone())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = 0
    while time.perf_counter() - t0 < t_hier:
        rec.run(10)
        its += 10
    torch.cuda.synchronize()
    t_flat = time.perf_counter() - t0
    F_f = rec.history["F"][-1]
    err_f = float((rec.psi - psi_true).norm() / psi_true.norm())
    h.close()
    per_level = [{"binning": r["b"], "iterations": len(r["history"]["F"]) - 1,
                  "F_first": r["history"]["F"][0], "F_last": r["history"]["F"][-1]}
                 for r in hier.results]
    return {"metric": "full-grid F after equal wall time, hierarchical vs flat reconstruction",
            "value": round(F_h, 4), "unit": "F2", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "hier: 16 angles of the medium workload (psi 512^2 on 1024^2, "
                                   "4 distances), noise-free, levels " + str(levels)},
            "hierarchical": {"seconds": round(t_hier, 3), "F_full_grid": F_h,
                             "rel_err_psi": err_h, "levels": per_level},
            "flat": {"seconds": round(t_flat, 3), "iterations": its, "F_full_grid": F_f,
                     "rel_err_psi": err_f}}


# ---------------------------------------------------------------- batch of reconstructions

def batch_specs(seed, count=64, budget_gb=280.0):
    """Seeded uneven batch: side n in {256, 384, 512, 1024, 2048}, 1-4 distances, 16-128
    angles, P = 2n (768 for n = 384: one radix-3 step), 16-angle chunks.  Planned device
    memory per instance: psi and grad_psi, data, q / grad_q / two P x P scratch fields, p_j,
    the per-plane slots of a chunk (box rows x n for Y and box rows x box columns for w, the
    box at most n + 16 per axis) and the plane tables.  Instances are dropped from the largest
    down if the plan exceeds the budget (280 GB of the GPU's 298 GB)."""
    rng = hs.rng_for(seed, 77)
    specs = []
    for i in range(count):
        n = int(rng.choice([256, 384, 512, 1024, 2048]))
        J = int(rng.integers(1, 5))
        K = int(rng.integers(16, 129))
        P = 2 * n
        chunk = min(K, 16)
        mem = (2 * K * n * n * 8 + K * J * n * n * 4 + 4 * P * P * 8 + J * P * P * 8
               + chunk * J * 2 * (n + 16) ** 2 * 8 + K * J * (2 * (n + 16) * 8 + 2 * n * 16)
               + 3 * n * n * 8)
        specs.append({"n": n, "P": P, "J": J, "K": K, "chunk": chunk, "mem": mem, "seed": i})
    kept = sorted(specs, key=lambda d: d["mem"])
    while sum(d["mem"] for d in kept) > budget_gb * 1e9:
        kept.pop()
    ids = {d["seed"] for d in kept}
    return [d for d in specs if d["seed"] in ids], len(specs) - len(kept)


def run_batch(args):
    import torch
    from paper_2407_20304_gb300 import Holo
    from paper_2407_20304_gb300.batch import HoloBatch, Instance
    import __graft_entry__
    __graft_entry__.build()
    g = hs.WORKLOAD_GEOMETRY
    specs, dropped = batch_specs(hs.SEED_BASE + 3000)
    insts = []
    for sp in specs:
        n, P, J, K, chunk = sp["n"], sp["P"], sp["J"], sp["K"], sp["chunk"]
        rng = hs.rng_for(hs.SEED_BASE + 3000, 1000 + sp["seed"])
        psi_true = torch.from_numpy(hs.transmittance(hs.ellipse_phase(n, rng)).astype(np.complex64)).cuda()
        q_true = torch.from_numpy(hs.striped_probe(P, 40.0 * n / 128, rng).astype(np.complex64)).cuda()
        t = hs.sample_shifts(K, J, rng).astype(np.float32)
        h = Holo(n, K, J, g["wavelength"], g["pixel"], g["Z"], g["z"][:J], pad=P, chunk=chunk)
        h.set_shifts(t)
        sqrt_d = torch.empty((K, J, n, n), dtype=torch.float32, device="cuda")
        ones_ref = torch.ones((n, n), dtype=torch.float32, device="cuda")
        h.set_data(sqrt_d, ones_ref)
        h.set_probe(q_true)
        gen = torch.Generator(device="cuda").manual_seed(sp["seed"])
        for k0 in range(0, K, chunk):
            nk = min(chunk, K - k0)
            u = torch.empty((nk, J, n, n), dtype=torch.complex64, device="cuda")
            h.forward(psi_true.expand(nk, n, n).contiguous(), k0=k0, u_out=u)
            inten = u.abs().square_()
            c = 1e4 / inten.mean()
            sqrt_d[k0:k0 + nk] = torch.poisson(inten * c, generator=gen).div_(c).sqrt_()
            del u, inten
        lo = P // 2 - n // 2
        _, zeta = derived(g["z"][:J], g["Z"])
        bref = h.propagate(q_true, zeta[0])[lo:lo + n, lo:lo + n]
        sqrt_dref = bref.abs().contiguous()
        h.set_data(sqrt_d, sqrt_dref)
        inst = Instance(h, torch.ones((K, n, n), dtype=torch.complex64, device="cuda"),
                        q_true.clone())
        inst.data = (sqrt_d, sqrt_dref)
        insts.append(inst)
        # the data-generation temporaries go back to the device before the next context
        # allocates its workspace
        torch.cuda.empty_cache()
    b = HoloBatch(insts)
    loop_ms = b.time_loop(reps=2)
    best_ms, sched, cost = b.autotune(candidates=(1, 2, 4, 8), reps=2)
    torch.cuda.synchronize()
    planes = b.planes
    return {
        "metric": "plane-gradient evals/s, batch of uneven reconstructions", "unit": UNIT,
        "value": round(planes / (best_ms / 1e3), 1), "n_gpus": 1, "ms_per_step": round(best_ms, 3),
        "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch: {len(insts)} instances (sides 256-2048, pad 2n, "
                               f"1-4 distances, 16-128 angles, 16-angle chunks)"
                               + (f", {dropped} largest dropped for the memory budget" if dropped else ""),
                   "planes_per_step": planes,
                   "sizes": sorted({s["n"] for s in specs})},
        "loop": {"value": round(planes / (loop_ms / 1e3), 1), "ms_per_step": round(loop_ms, 3)},
        "graph": {"branches": len(sched), "ms_per_step": round(best_ms, 3),
                  "tuning": {str(k): round(v["ms"], 3) for k, v in b.tuning.items()}},
    }


def main():
    args = parse()
    if args.workload == "batch":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.workload == "recon":
        print(json.dumps(run_recon(args)), flush=True)
        return
    if args.workload == "hier":
        print(json.dumps(run_hier(args)), flush=True)
        return
    w = hs.workloads()[args.workload]
    if args.chunk:
        import dataclasses
        w = dataclasses.replace(w, chunk=args.chunk)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, w)), flush=True)
        return
    import torch
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        tdist.barrier()
        __graft_entry__.build()
    result, h = run_ours(args, w, rank, world, local_rank)
    h.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"], result["err_vs_fp64"] = cpu_baseline(w, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
