"""FP64 nonlinear conjugate gradients (Sec. 2): the Dai-Yuan direction of Eq. DaiYuan2 and
the Fletcher-Reeves / Polak-Ribiere-Polyak formulas the paper names beside it.

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


def fletcher_reeves_beta(g_new, g_old):
    """beta_FR = ||g_new||^2 / ||g_old||^2 (Fletcher-Reeves, named in Sec. 2); None if
    g_old = 0."""
    den = re_inner(g_old, g_old)
    return re_inner(g_new, g_new) / den if den > 0.0 else None


def polak_ribiere_beta(g_new, g_old):
    """beta_PRP = Re <g_new, g_new - g_old> / ||g_old||^2 (Polak-Ribiere-Polyak, named in
    Sec. 2); None if g_old = 0."""
    den = re_inner(g_old, g_old)
    return (re_inner(g_new, g_new) - re_inner(g_new, g_old)) / den if den > 0.0 else None


def direction(g_new, g_old, eta, rule="dai-yuan"):
    """Next CG direction -g_new + beta eta for rule 'dai-yuan' (Eq. DaiYuan2),
    'fletcher-reeves' or 'polak-ribiere'.  Dai-Yuan restarts (-g_new) when its denominator
    is not positive (reading R7); the other two restart when beta is undefined or the new
    direction is not a descent direction (Re <g_new, eta_new> >= 0)."""
    if rule == "dai-yuan":
        return dai_yuan_direction(g_new, g_old, eta)
    beta = fletcher_reeves_beta(g_new, g_old) if rule == "fletcher-reeves" else \
        polak_ribiere_beta(g_new, g_old)
    if beta is None:
        return -g_new, 0.0
    e = -g_new + beta * eta
    if not re_inner(g_new, e) < 0.0:
        return -g_new, 0.0
    return e, beta


def armijo(f, f0, slope, x, eta, gamma0, max_halvings, c=1e-4):
    """Largest gamma in {gamma0 / 2^i} (i <= max_halvings) with the sufficient decrease
    f(x + gamma eta) <= f0 + c gamma slope, slope = Re <grad f(x), eta> < 0.

    Returns (gamma, f_new); gamma = 0 and f_new = f0 when no trial qualifies or eta is not a
    descent direction."""
    if not slope < 0.0:
        return 0.0, f0
    gamma = gamma0
    for _ in range(max_halvings + 1):
        fx = f(x + gamma * eta)
        if fx <= f0 + c * gamma * slope:
            return gamma, fx
        gamma *= 0.5
    return 0.0, f0


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
                max_halvings=20, update_q=True, rule="dai-yuan", line_search="backtracking",
                probe_shifts=None):
    """Joint psi / q reconstruction by nonlinear conjugate gradients (Sec. 2).

    rule: the direction formula ('dai-yuan' of Eq. DaiYuan2, 'fletcher-reeves',
    'polak-ribiere'); line_search: 'backtracking' (first decrease of F, reading R7) or
    'armijo' (sufficient decrease with c = 1e-4).  Returns a dict with the final psi, q and
    per-iteration F, gamma_psi, gamma_q, beta_psi, beta_q.  The initial trial step of each
    block is twice its last accepted step (gamma0 at the first iteration).  probe_shifts:
    the s_kj of Eq. min1 (reading R5 of oracle.holo), or None.
    """
    ps = probe_shifts
    psi = np.array(psi0, dtype=np.complex128)
    q = np.array(q0, dtype=np.complex128)
    F, gpsi, gq = holo.gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo, ps)
    eta_psi, eta_q = -gpsi, -gq
    trial_psi = trial_q = gamma0
    hist = {"F": [F], "gamma_psi": [], "gamma_q": [], "beta_psi": [], "beta_q": [],
            "F_after_psi": []}

    def search(f, F0, g, x, eta, trial):
        if line_search == "armijo":
            return armijo(f, F0, re_inner(g, eta), x, eta, trial, max_halvings)
        return backtrack(f, F0, x, eta, trial, max_halvings)

    for _ in range(iters):
        def f_psi(x):
            return holo.functional(x, q, shifts, sqrt_d, sqrt_dref, geo, ps)
        gam_psi, F = search(f_psi, F, gpsi, psi, eta_psi, trial_psi)
        psi = psi + gam_psi * eta_psi
        hist["F_after_psi"].append(F)
        gam_q = 0.0
        if update_q:
            def f_q(x):
                return holo.functional(psi, x, shifts, sqrt_d, sqrt_dref, geo, ps)
            # the q gradient at the updated psi is not evaluated; the slope of the Armijo
            # test uses the gradient of the last evaluation
            gam_q, F = search(f_q, F, gq, q, eta_q, trial_q)
            q = q + gam_q * eta_q
        trial_psi = 2.0 * gam_psi if gam_psi > 0 else trial_psi
        trial_q = 2.0 * gam_q if gam_q > 0 else trial_q
        F_new, gpsi_new, gq_new = holo.gradients(psi, q, shifts, sqrt_d, sqrt_dref, geo, ps)
        eta_psi, b_psi = direction(gpsi_new, gpsi, eta_psi, rule)
        eta_q, b_q = direction(gq_new, gq, eta_q, rule)
        gpsi, gq, F = gpsi_new, gq_new, F_new
        hist["F"].append(F)
        hist["gamma_psi"].append(gam_psi)
        hist["gamma_q"].append(gam_q)
        hist["beta_psi"].append(b_psi)
        hist["beta_q"].append(b_q)
    return {"psi": psi, "q": q, "hist": hist}


def reconstruct_hierarchical(sqrt_d, sqrt_dref, shifts, geo, levels, q0=None,
                             probe_shifts=None, **kw):
    """Hierarchical reconstruction (Sec. 3, on speeding up): for each (b, iters) of `levels`,
    from the coarsest binning b to b = 1, run `reconstruct` on data binned by b (pixel b dx,
    side n/b on a P/b grid, shifts t/b and probe shifts s/b), starting from psi = 1 and the
    initial probe of the binned reference image at the first level and from the previous
    level's psi and q upsampled twice as dense afterwards.  Returns the list of per-level
    results."""
    import dataclasses
    out = []
    psi = q = None
    for i, (b, iters) in enumerate(levels):
        g = dataclasses.replace(geo, n=geo.n // b, P=geo.P // b, pixel=geo.pixel * b)
        d = holo.bin_amplitudes(sqrt_d, b)
        dr = holo.bin_amplitudes(sqrt_dref, b) if sqrt_dref is not None else None
        t = np.asarray(shifts, np.float64) / b
        s = None if probe_shifts is None else np.asarray(probe_shifts, np.float64) / b
        if i == 0:
            psi = np.ones((d.shape[0], g.n, g.n), np.complex128)
            q = holo.initial_probe(dr, g) if q0 is None else q0
        else:
            factor = levels[i - 1][0] // b
            while factor > 1:
                psi, q = holo.upsample2(psi), holo.upsample2(q)
                factor //= 2
        res = reconstruct(psi, q, t, d, dr, g, iters, probe_shifts=s, **kw)
        psi, q = res["psi"], res["q"]
        out.append({"b": b, "psi": psi, "q": q, "hist": res["hist"]})
    return out
