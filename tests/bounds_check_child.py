"""Child process of tests/test_gpu_bounds_check.py: evaluates the gradients of the problems in
an .npz with the library the environment selects (HOLO_BOUNDS_CHECK=1: the bounds-checking
build) and writes loss, grad_psi and grad_q to another .npz.  Then writes bit 2 of the device
error word from the host and records the status the next loss read returns.

    python tests/bounds_check_child.py IN.npz OUT.npz
"""

import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2407_20304_gb300 import Holo, HoloError, _lib  # noqa: E402


def main(src, dst):
    d = np.load(src)
    out = {"lib_path": np.array(_lib.LIB_PATH)}
    for p in json.loads(str(d["problems"])):
        key = p["key"]
        h = Holo(p["n"], p["K"], p["J"], p["wavelength"], p["pixel"], p["Z"], p["z"], pad=p["P"])
        if key + "_s" in d:  # probe shifts first: the plane boxes follow from them
            h.set_probe_shifts(d[key + "_s"].astype(np.float32))
        h.set_shifts(d[key + "_t"].astype(np.float32))
        h.set_data(torch.from_numpy(d[key + "_sqrt_d"].astype(np.float32)).cuda(),
                   torch.from_numpy(d[key + "_sqrt_dref"].astype(np.float32)).cuda())
        h.set_probe(torch.from_numpy(d[key + "_q"].astype(np.complex64)).cuda())
        loss, gp, gq = h.gradient(torch.from_numpy(d[key + "_psi"].astype(np.complex64)).cuda())
        out[key + "_loss"] = np.array(loss)
        out[key + "_gp"] = gp.cpu().numpy()
        out[key + "_gq"] = gq.cpu().numpy()
        h.close()
    # the status of a failed device check, written from the host (bit 2 of the error word)
    p = json.loads(str(d["problems"]))[0]
    key = p["key"]
    h = Holo(p["n"], p["K"], p["J"], p["wavelength"], p["pixel"], p["Z"], p["z"], pad=p["P"])
    h.set_shifts(d[key + "_t"].astype(np.float32))
    h.set_data(torch.from_numpy(d[key + "_sqrt_d"].astype(np.float32)).cuda(),
               torch.from_numpy(d[key + "_sqrt_dref"].astype(np.float32)).cuda())
    h.set_probe(torch.from_numpy(d[key + "_q"].astype(np.complex64)).cuda())
    psi = torch.from_numpy(d[key + "_psi"].astype(np.complex64)).cuda()
    h.set_device_error(2)
    status = 0
    try:
        h.gradient(psi)
    except HoloError as e:
        status = e.status
    out["bounds_status"] = np.array(status)
    # cleared by that read: the next evaluation is fine
    out["after_loss"] = np.array(h.gradient(psi)[0])
    h.close()
    np.savez(dst, **out)


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
