"""Host-side models of bench.py: the per-pass algorithmic byte model behind the roofline
numerator, the batch memory plan, and the rule that recorded DRAM traffic is used only for the
kernel sources it was measured on."""

import json

import numpy as np
import pytest

import bench
import holo_synth as hs


def _large_boxes():
    w = hs.workloads()["large"]
    g = hs.WORKLOAD_GEOMETRY
    mt, _ = bench.derived(g["z"][:w.n_dist], g["Z"])
    t = hs.sample_shifts(w.chunk, w.n_dist, hs.rng_for(1, 2))
    return w, bench.boxes(w.n, w.P, mt, t)


def test_box_model_bounds_the_resample_support():
    """Each box covers every P-grid position whose bilinear taps reach psi (xi in (-1, n)) and
    stays inside the grid; at m~ = 1 it is n plus a few pixels."""
    w, box = _large_boxes()
    n, P = w.n, w.P
    g = hs.WORKLOAD_GEOMETRY
    mt, _ = bench.derived(g["z"][:w.n_dist], g["Z"])
    for j in range(w.n_dist):
        sy, _ = box[0][j]
        support = n / mt[j] + 1 / mt[j]
        assert support <= sy <= support + 5 and sy <= P
    assert n + 1 <= box[0][0][0] <= n + 6


def test_algorithmic_bytes_per_plane_of_the_large_workload():
    """Per plane at psi 2048^2 / pad 4096 (s box rows, s_x box columns): pass A 8n^2 + 16 s s_x
    + 8 s n, pass B 16 s n + 4 n^2 (+ 24 n^2 per launch), pass C 16 s n + 24 s s_x, pass D 8 s n
    (+ 8 n^2 per angle): about 106, 71, 121 and 35 MB."""
    w, box = _large_boxes()
    n, planes = w.n, w.chunk * w.n_dist
    c = bench.algorithmic_costs(n, w.P, box)
    per = {k: v["bytes"] / planes / 1e6 for k, v in c.items()}
    assert per["pass_a"] == pytest.approx(106, abs=1.5)
    assert per["pass_b"] == pytest.approx(71, abs=0.5)
    assert per["pass_c"] == pytest.approx(121, abs=1.5)
    assert per["pass_d"] == pytest.approx(35, abs=0.5)
    sb = sum(16 * sy * n + 4 * n * n for row in box for sy, _ in row) + 24 * n * n
    assert c["pass_b"]["bytes"] == sb
    # pass B: four length-P transforms per detector column and plane dominate its flops
    fft = 5.0 * w.P * np.log2(w.P)
    assert c["pass_b"]["flops"] > planes * n * 4 * fft


def test_full_grid_boxes_cost_more_than_the_support_boxes():
    w, box = _large_boxes()
    full = [[(w.P, w.P)] * w.n_dist] * w.chunk
    a, b = bench.algorithmic_costs(w.n, w.P, box), bench.algorithmic_costs(w.n, w.P, full)
    for k in ("pass_a", "pass_c"):
        assert b[k]["bytes"] > 2 * a[k]["bytes"] and b[k]["flops"] > 2 * a[k]["flops"]


def test_batch_plan_keeps_all_instances_within_the_budget():
    specs, dropped = bench.batch_specs(hs.SEED_BASE + 3000)
    assert dropped == 0 and len(specs) == 64
    assert sum(d["mem"] for d in specs) <= 280e9
    assert {d["n"] for d in specs} == {256, 384, 512, 1024, 2048}
    assert all(d["P"] == 2 * d["n"] and 1 <= d["J"] <= 4 and 16 <= d["K"] <= 128 for d in specs)
    small, dropped_small = bench.batch_specs(hs.SEED_BASE + 3000, budget_gb=150.0)
    assert dropped_small > 0 and sum(d["mem"] for d in small) <= 150e9
    kept = {d["seed"] for d in small}
    gone = [d for d in specs if d["seed"] not in kept]
    assert min(d["mem"] for d in gone) >= max(d["mem"] for d in small)


def test_recorded_traffic_only_for_the_measured_sources(tmp_path, monkeypatch):
    rec = {"pass_b": {"kernel_hash": "abc", "n": 2048, "full_launch_planes": 240,
                      "bytes_per_launch_full": 1.5e10}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "abc")
    assert bench.recorded_traffic("pass_b", 2048, 240) == 1.5e10
    assert bench.recorded_traffic("pass_b", 1024, 240) is None
    assert bench.recorded_traffic("pass_b", 2048, 64) is None
    assert bench.recorded_traffic("pass_a", 2048, 240) is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "changed")
    assert bench.recorded_traffic("pass_b", 2048, 240) is None
