"""The synthetic configurations 0 .. 4 (holo_synth/configs.json): their order and sizes, the
workloads built from them, the library geometry they map to, and the batch's ranges."""

import holo_synth as hs


def test_five_configs_in_order():
    names = [hs.config(i)["name"] for i in range(5)]
    assert names == ["tiny", "medium", "autograd", "batch", "large"]
    for i in range(5):
        assert hs.config(i) == hs.config(names[i])


def test_workloads_from_the_configs():
    w = hs.workloads()
    assert sorted(w) == ["autograd", "large", "medium", "tiny"]
    assert (w["tiny"].n, w["tiny"].P, w["tiny"].n_angles, w["tiny"].n_dist) == (128, 256, 8, 4)
    assert (w["medium"].n, w["medium"].P, w["medium"].n_angles, w["medium"].chunk) == (512, 1024, 180, 180)
    assert (w["autograd"].n, w["autograd"].P, w["autograd"].n_angles) == (1024, 2048, 90)
    assert (w["large"].n, w["large"].P, w["large"].n_angles, w["large"].chunk) == (2048, 4096, 900, 60)
    assert w["tiny"].counts == 0.0 and all(w[k].counts == 1e4 for k in ("medium", "autograd", "large"))
    assert len({x.seed for x in w.values()}) == 4


def test_holo_geometry_fields():
    g = hs.holo_geometry("large")
    assert (g["n"], g["pad"], g["n_angles"], g["n_dist"], g["chunk"]) == (2048, 4096, 900, 4, 60)
    assert tuple(g["z"]) == hs.WORKLOAD_GEOMETRY["z"]
    assert g["w_ref"] == 1.0 and g["ext"] == 1.0
    assert hs.holo_geometry(0, chunk=4)["chunk"] == 4
    try:
        hs.holo_geometry("batch")
        raise AssertionError("the batch has no single geometry")
    except ValueError:
        pass


def test_batch_ranges_match_its_generator():
    import bench
    c = hs.config("batch")
    specs, _ = bench.batch_specs(c["seed"], count=c["count"], budget_gb=c["budget_gb"])
    assert {s["n"] for s in specs} <= set(c["sides"])
    assert all(c["n_dist"][0] <= s["J"] <= c["n_dist"][1] for s in specs)
    assert all(c["n_angles"][0] <= s["K"] <= c["n_angles"][1] for s in specs)
    assert all(s["P"] == 2 * s["n"] and s["chunk"] == min(s["K"], c["chunk"]) for s in specs)
