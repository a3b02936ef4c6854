"""Failure paths of the library, driven from the host (nothing faults, traps or hangs on the
GPU): the device error word that a bounded wait sets when it gives up, injected allocation,
argument and numeric failures (HOLO_FAULT), and non-finite data.  After each failure the
context stays usable and the next call gives the clean result bit for bit."""

import numpy as np
import pytest

import holo_synth as hs
from oracle import holo as oh

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
G = hs.WORKLOAD_GEOMETRY


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    n, P, K, J = 64, 128, 2, 4
    rng = hs.rng_for(hs.SEED_BASE + 31, 0)
    geo = oh.Geometry(G["wavelength"], G["pixel"], G["Z"], G["z"], n, P)
    w = hs.Workload("f", n, P, K, J, "ellipses", 20.0, 0.0, K, 0)
    psi_true = hs.object_stack(w, range(K), rng)
    q = hs.striped_probe(P, 20.0, rng)
    t = hs.sample_shifts(K, J, rng).astype(np.float32)
    sqrt_d = np.abs(oh.forward(psi_true, q, t.astype(np.float64), geo)).astype(np.float32)
    sqrt_dref = np.abs(oh.reference_field(q, geo)).astype(np.float32)
    psi = hs.perturbed_probe(psi_true, rng, 0.05).astype(np.complex64)
    return dict(n=n, P=P, K=K, J=J, t=t, sqrt_d=sqrt_d, sqrt_dref=sqrt_dref, q=q.astype(np.complex64),
                psi=psi)


def _holo(s):
    from paper_2407_20304_gb300 import Holo
    h = Holo(s["n"], s["K"], s["J"], G["wavelength"], G["pixel"], G["Z"], G["z"], pad=s["P"])
    h.set_shifts(s["t"])
    h.set_data(torch.from_numpy(s["sqrt_d"]).cuda(), torch.from_numpy(s["sqrt_dref"]).cuda())
    h.set_probe(torch.from_numpy(s["q"]).cuda())
    return h


def test_device_error_word_reports_timeout_once(setup):
    from paper_2407_20304_gb300 import HoloError
    h = _holo(setup)
    psi = torch.from_numpy(setup["psi"]).cuda()
    clean = h.gradient(psi)
    h.set_device_error(1)
    with pytest.raises(HoloError, match="TIMEOUT") as e:
        h.gradient(psi)
    assert e.value.status == 4
    again = h.gradient(psi)          # the word was cleared by the failing read
    assert again[0] == clean[0]
    assert torch.equal(again[1], clean[1]) and torch.equal(again[2], clean[2])
    # a forward call reads the word too; clearing it by hand leaves nothing to report
    h.set_device_error(5)
    with pytest.raises(HoloError, match="TIMEOUT"):
        h.forward(psi)
    h.set_device_error(5)
    h.set_device_error(0)
    assert h.forward(psi) == h.forward(psi)
    # bit 2 is a failed device bounds check, reported before a wait that gave up
    for word in (2, 3):
        h.set_device_error(word)
        with pytest.raises(HoloError, match="BOUNDS") as e:
            h.gradient(psi)
        assert e.value.status == 8
    assert h.gradient(psi)[0] == clean[0]
    h.close()


def test_injected_host_faults(setup, monkeypatch):
    from paper_2407_20304_gb300 import Holo, HoloError
    s = setup
    psi = torch.from_numpy(s["psi"]).cuda()
    monkeypatch.setenv("HOLO_FAULT", "alloc")
    with pytest.raises(HoloError, match="OOM"):
        Holo(s["n"], s["K"], s["J"], G["wavelength"], G["pixel"], G["Z"], G["z"], pad=s["P"])
    monkeypatch.delenv("HOLO_FAULT")
    h = _holo(s)
    clean = h.gradient(psi)
    for kind, status in (("arg", "ARG"), ("nan", "NUMERIC")):
        monkeypatch.setenv("HOLO_FAULT", kind)
        with pytest.raises(HoloError, match=status):
            h.gradient(psi)
        monkeypatch.delenv("HOLO_FAULT")
        again = h.gradient(psi)
        assert again[0] == clean[0] and torch.equal(again[1], clean[1])
    h.close()


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_data_is_reported(setup, bad):
    from paper_2407_20304_gb300 import HoloError
    s = dict(setup)
    d = s["sqrt_d"].copy()
    d[1, 2, 10, 20] = bad
    s["sqrt_d"] = d
    h = _holo(s)
    with pytest.raises(HoloError, match="NUMERIC"):
        h.gradient(torch.from_numpy(s["psi"]).cuda())
    h.close()


def test_checkpoint_resume_on_the_gpu_is_bit_exact(setup, tmp_path):
    """The GPU driver saved after 2 iterations and resumed in a fresh driver (and a fresh
    context) continues bit for bit as an uninterrupted 4-iteration run: every kernel reduces
    in a fixed order."""
    from paper_2407_20304_gb300.cg import Reconstruction
    s = setup
    q0 = torch.from_numpy(s["q"]).cuda()
    psi0 = torch.ones((s["K"], s["n"], s["n"]), dtype=torch.complex64, device="cuda")
    full = Reconstruction(_holo(s), psi0.clone(), q0.clone())
    full.run(4)
    part = Reconstruction(_holo(s), psi0.clone(), q0.clone())
    part.run(2)
    path = tmp_path / "gpu_state.npz"
    part.save(path)
    res = Reconstruction(_holo(s), torch.zeros_like(psi0), torch.zeros_like(q0))
    res.load(path)
    res.run(2)
    assert res.history == full.history
    assert torch.equal(res.psi, full.psi) and torch.equal(res.q, full.q)
