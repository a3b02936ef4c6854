"""Sanity of the seeded input generators (shapes, ranges, determinism)."""

import numpy as np

import holo_synth as hs


def test_layered_cube_phase_range_and_structure():
    rng = hs.rng_for(hs.SEED_BASE, 3)
    cube = hs.LayeredCube(256, rng)
    for th in (0.0, 0.3, np.pi / 4, 1.2):
        ph = cube.phase(th)
        assert ph.shape == (256, 256)
        assert np.all(ph <= 1e-12)
        assert ph.min() >= -np.pi * 1.5
    assert cube.phase(np.pi / 4).min() == np.float64(-np.pi) or \
        abs(cube.phase(np.pi / 4).min() + np.pi) < 1e-9
    # empty corners (outside the cube) are free space
    assert cube.phase(0.0)[0, 0] == 0.0
    # layers: the projected phase is not constant across the cube
    ph = cube.phase(0.0)[128]
    assert len(np.unique(np.round(ph[ph < 0], 6))) > 4


def test_transmittance_and_probe():
    rng = hs.rng_for(hs.SEED_BASE, 4)
    w = hs.workloads()["tiny"]
    psi = hs.object_stack(w, range(2), rng)
    assert psi.shape == (2, 128, 128) and np.all(np.isfinite(psi))
    assert np.all(np.abs(psi) <= 1.0 + 1e-12)
    q = hs.striped_probe(256, 40.0, rng)
    assert q.shape == (256, 256) and np.all(np.isfinite(q))
    assert np.abs(q[128, 128]) > 0.3 and np.abs(q[0, 0]) < 1e-3


def test_generators_are_seeded():
    a = hs.sample_shifts(3, 4, hs.rng_for(5, 1))
    b = hs.sample_shifts(3, 4, hs.rng_for(5, 1))
    c = hs.sample_shifts(3, 4, hs.rng_for(5, 2))
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert np.all(np.abs(a) <= 2.0)


def test_poisson_amplitude_mean_counts():
    rng = hs.rng_for(7, 0)
    inten = np.full((200, 200), 0.25)
    amp = hs.poisson_amplitude(inten, 1e4, rng)
    assert abs(np.mean(amp ** 2) - 0.25) < 1e-3
    np.testing.assert_array_equal(hs.poisson_amplitude(inten, 0, rng), 0.5)


def test_workloads_have_the_stated_shapes():
    """psi side, padded grid, angles, distances, chunk, probe sigma (40 px at n = 128, scaled
    with n) and Poisson counts of the synthetic workloads."""
    w = hs.workloads()
    expect = {"tiny": (128, 256, 8, 4, 8, 0.0, "ellipses"),
              "medium": (512, 1024, 180, 4, 180, 1e4, "layers"),
              "autograd": (1024, 2048, 90, 4, 90, 1e4, "layers"),
              "large": (2048, 4096, 900, 4, 60, 1e4, "layers")}
    for name, (n, P, K, J, chunk, counts, phantom) in expect.items():
        x = w[name]
        assert (x.n, x.P, x.n_angles, x.n_dist, x.chunk, x.counts, x.phantom) == \
            (n, P, K, J, chunk, counts, phantom)
        assert x.probe_sigma == 40.0 * n / 128
    assert len({x.seed for x in w.values()}) == len(w)
    g = hs.WORKLOAD_GEOMETRY
    assert g["wavelength"] == 3.72e-11 and g["pixel"] == 10e-9
    assert tuple(g["z"]) == (4.6e-4, 5.1e-4, 6.2e-4, 8.3e-4)
