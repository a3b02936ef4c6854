"""The HOLO_BOUNDS_CHECK build (device checks of table-driven indices that report
HOLO_ERR_BOUNDS instead of faulting): built here, run in a child process that loads it
(HOLO_BOUNDS_CHECK=1), its results against the normal build and the FP64 oracle.  A failed
check is produced on the host only (bit 2 of the device error word): nothing is given an
out-of-range index on the GPU."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import holo as oh
from test_gpu_parity import GRAD_TOL, LOSS_TOL, dev, make_holo, make_problem, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# line lengths 2^k and 3 * 2^k, the n = P/2 forms with the TMA stage, the P = 4096 engine with
# its middle-half forms, and the probe-shift forms (full-grid boxes)
CASES = [("a", 64, 128, 2, 4, "start"), ("b", 384, 768, 2, 4, "object"),
         ("c", 1024, 2048, 1, 4, "object"), ("d", 2048, 4096, 1, 2, "object"),
         ("e", 96, 192, 2, 4, "object")]
SHIFTED = {"e"}


def _probe_shifts(key, K, J):
    rng = np.random.default_rng(ord(key))
    return rng.uniform(-2.0, 2.0, (K, J, 2))


@pytest.fixture(scope="module")
def child_run(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_20304_gb300 import build
    build.build(bounds_check=True)
    tmp = tmp_path_factory.mktemp("bc")
    arrays, problems, prs = {}, [], {}
    for key, n, P, K, J, point in CASES:
        pr = make_problem(n, P, K, J=J, seed=13 * n + J, point=point)
        prs[key] = pr
        geo = pr["geo"]
        problems.append(dict(key=key, n=n, P=P, K=K, J=J, wavelength=geo.wavelength,
                             pixel=geo.pixel, Z=geo.Z, z=list(geo.z)))
        arrays.update({key + "_t": pr["t"], key + "_sqrt_d": pr["sqrt_d"],
                       key + "_sqrt_dref": pr["sqrt_dref"], key + "_q": pr["q"],
                       key + "_psi": pr["psi"]})
        if key in SHIFTED:
            # rounded to float32 as the library takes them, so both sides see the same shifts
            pr["s"] = _probe_shifts(key, K, J).astype(np.float32).astype(np.float64)
            arrays[key + "_s"] = pr["s"]
    src, dst = tmp / "in.npz", tmp / "out.npz"
    np.savez(src, problems=np.array(json.dumps(problems)), **arrays)
    env = dict(os.environ, HOLO_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_check_child.py"),
                        str(src), str(dst)], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return prs, np.load(dst)


def test_child_loaded_the_bounds_checking_build(child_run):
    _, out = child_run
    assert str(out["lib_path"]).endswith(os.path.join("_build_bc", "libholo.so"))


@pytest.mark.parametrize("key", [c[0] for c in CASES])
def test_bounds_checking_build_matches_the_normal_build_and_the_oracle(child_run, key):
    prs, out = child_run
    pr = prs[key]
    s = pr.get("s")
    if s is None:
        h = make_holo(pr)
    else:
        # probe shifts first: the plane boxes follow from them
        from paper_2407_20304_gb300 import Holo
        geo = pr["geo"]
        h = Holo(geo.n, pr["psi"].shape[0], geo.n_dist, geo.wavelength, geo.pixel, geo.Z, geo.z,
                 pad=geo.P, w_ref=geo.w_ref, ext=geo.ext)
        h.set_probe_shifts(s.astype(np.float32))
        h.set_shifts(pr["t"].astype(np.float32))
        h.set_data(dev(pr["sqrt_d"], torch.float32), dev(pr["sqrt_dref"], torch.float32))
        h.set_probe(dev(pr["q"], torch.complex64))
    loss, gp, gq = h.gradient(dev(pr["psi"], torch.complex64))
    gp, gq = gp.cpu().numpy(), gq.cpu().numpy()
    # the checks change no arithmetic: the same results as the normal build
    assert abs(float(out[key + "_loss"]) - loss) <= 1e-12 * abs(loss)
    assert rel(out[key + "_gp"], gp) <= 1e-6 and rel(out[key + "_gq"], gq) <= 1e-6
    F, gp_ref, gq_ref = oh.gradients(pr["psi"], pr["q"], pr["t"], pr["sqrt_d"], pr["sqrt_dref"],
                                     pr["geo"], s)
    assert abs(float(out[key + "_loss"]) - F) / F < LOSS_TOL
    assert rel(out[key + "_gp"], gp_ref) < GRAD_TOL and rel(out[key + "_gq"], gq_ref) < GRAD_TOL
    h.close()


def test_a_failed_check_reads_as_holo_err_bounds(child_run):
    _, out = child_run
    assert int(out["bounds_status"]) == 8          # HOLO_ERR_BOUNDS
    assert np.isfinite(float(out["after_loss"]))    # the read cleared the word
