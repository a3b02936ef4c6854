"""FP64 nonlinear conjugate gradients with the Dai-Yuan direction (Sec. 2, Eq. DaiYuan2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading R7 (the paper names "a line-search procedure" that guarantees
F^(m+1) <= F^(m), and does not say whether psi and q share the step):

* psi and q each keep their own Dai-Yuan direction, built from FP64 real inner products
  <a, b> = Re sum conj(a) b;  eta^(0) = -g^(0).
* After one shared gradient evaluation the step length of psi is found by halving a
  trial step until F decreases, then the step length of q the same way from the
  updated psi.  A block whose trials never decrease F gets step 0 (the "gaps" of
  Fig. conv), so F never increases.
* A non-positive Dai-Yuan denominator restarts that block with eta = -g.
"""

import numpy as np

from . import holo


def re_inner(a, b):
    """Re <a, b> = Re sum conj(a) b, accumulated in FP64."""
    return float(np.real(np.vdot(np.asarray(a, np.complex128), np.asarray(b, np.complex128))))


def dai_yuan_beta(g_new, g_old, eta):
    """beta = ||g_new||^2 / Re <g_new - g_old, eta>  (Eq. DaiYuan2).

    Returns None when the denominator is not positive (caller restarts with -g).
    """
    den = re_inner(g_new, eta) - re_inner(g_old, eta)
    if not den > 0.0:
        return None
    return re_inner(g_new, g_new) / den


def dai_yuan_direction(g_new, g_old, eta):
    """eta_new = -g_new + beta_DY eta (restart with -g_new if beta is undefined)."""
    beta = dai_yuan_beta(g_new, g_old, eta)
    if beta is None:
        return -g_new, 0.0
    return -g_new + beta * eta, beta


def backtrack(f, f0, x, eta, gamma0, max_halvings):
    """Largest gamma in {gamma0 / 2^i} (i <= max_halvings) with f(x + gamma eta) < f0.

    Returns (gamma, f_new); gamma = 0 and f_new = f0 when no trial decreases f.
    """
    gamma = gamma0
    for _ in range(max_halvings + 1):
        fx = f(x + gamma * eta)
        if fx < f0:
            return gamma, fx
        gamma *= 0.5
    return 0.0, f0


def reconstruct(psi0, q0, shifts, sqrt_d, sqrt_dref, geo, iters, gamma0=1.0,
                max_halvings=20, update_q=True):
    """Joint psi / q reconstruction by DY conjugate gradients (Sec. 2).

    Returns a dict with the final psi, q and per-iteration F, gamma_psi, gamma_q.
    The initial trial step of each block is twice its last accepted step (gamma0 at
    the first iteration).
    """
    psi = np.array(psi0, dtype=np.complex128)
    q = np.array(q0, dtype=np.complex128)
    F, gpsi, gq = holo.gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo)
    eta_psi, eta_q = -gpsi, -gq
    trial_psi = trial_q = gamma0
    hist = {"F": [F], "gamma_psi": [], "gamma_q": [], "beta_psi": [], "beta_q": [],
            "F_after_psi": []}
    for _ in range(iters):
        def f_psi(x):
            return holo.functional(x, q, shifts, sqrt_d, sqrt_dref, geo)
        gam_psi, F = backtrack(f_psi, F, psi, eta_psi, trial_psi, max_halvings)
        psi = psi + gam_psi * eta_psi
        hist["F_after_psi"].append(F)
        gam_q = 0.0
        if update_q:
            def f_q(x):
                return holo.functional(psi, x, shifts, sqrt_d, sqrt_dref, geo)
            gam_q, F = backtrack(f_q, F, q, eta_q, trial_q, max_halvings)
            q = q + gam_q * eta_q
        trial_psi = 2.0 * gam_psi if gam_psi > 0 else trial_psi
        trial_q = 2.0 * gam_q if gam_q > 0 else trial_q
        F_new, gpsi_new, gq_new = holo.gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo)
        eta_psi, b_psi = dai_yuan_direction(gpsi_new, gpsi, eta_psi)
        eta_q, b_q = dai_yuan_direction(gq_new, gq, eta_q)
        gpsi, gq, F = gpsi_new, gq_new, F_new
        hist["F"].append(F)
        hist["gamma_psi"].append(gam_psi)
        hist["gamma_q"].append(gam_q)
        hist["beta_psi"].append(b_psi)
        hist["beta_q"].append(b_q)
    return {"psi": psi, "q": q, "hist": hist}
