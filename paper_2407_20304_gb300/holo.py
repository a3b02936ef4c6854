"""Python binding of the C ABI: argument marshalling only.

`Holo` wraps one holo_ctx.  Device arrays are torch tensors (complex64 / float32,
contiguous, on the context's CUDA device); every computation runs in libholo.so on the
current torch stream at construction time.  Names follow the paper's notation: psi
(per-angle transmittances), q (probe), shifts t_kj, sqrt_d = sqrt(d~_kj).
"""

import ctypes

import numpy as np

from . import _lib


def _check(lib, ctx, status, where):
    if status != 0:
        detail = lib.holo_last_error(ctx).decode() if ctx else ""
        raise _lib.HoloError(status, where, detail)


def _ptr(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype, shape, name):
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise TypeError(f"{name} must be a C-contiguous numpy array of {dtype}")
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(a.shape)}")
    return ctypes.c_void_p(a.ctypes.data)


def dot_noalloc(a, b, stream=None):
    """Re <a, b> through holo_dot_noalloc: no context and no device allocation.

    For callers that must not allocate device memory; the partial sums live in a fixed
    device array of the library, so len(a) <= 2**28.  Calls that overlap on the GPU race.
    """
    import ctypes as ct

    import torch
    lib = _lib.load()
    if a.shape != b.shape:
        raise ValueError("shape mismatch")
    if a.numel() > _lib.NOALLOC_MAX_ELEMENTS:
        raise ValueError(f"dot_noalloc handles at most {_lib.NOALLOC_MAX_ELEMENTS} elements")
    pa = _ptr(a, torch.complex64, None, "a")
    pb = _ptr(b, torch.complex64, None, "b")
    if b.device != a.device:
        raise ValueError(f"a and b must be on one device, got {a.device} and {b.device}")
    # the library uses the scratch array of the current device: make a's device current
    with torch.cuda.device(a.device):
        s = stream if stream is not None else torch.cuda.current_stream(a.device)
        if s.device != a.device:
            raise ValueError(f"stream of {s.device} for tensors on {a.device}")
        out = ct.c_double(0.0)
        st = lib.holo_dot_noalloc(pa, pb, a.numel(), ct.byref(out), ct.c_void_p(s.cuda_stream))
    _check(lib, None, st, "holo_dot_noalloc")
    return out.value


def bin_amplitudes(a, b, stream=None):
    """Amplitudes [..., n, n] (float32 CUDA) binned by b: sqrt of the mean intensity of each
    b x b block (holo_bin_amplitudes)."""
    import torch
    n = a.shape[-1]
    if a.shape[-2] != n or n % b:
        raise ValueError("square images with a side divisible by b")
    out = torch.empty(a.shape[:-2] + (n // b, n // b), dtype=torch.float32, device=a.device)
    pa = _ptr(a, torch.float32, None, "a")
    s = stream if stream is not None else torch.cuda.current_stream(a.device)
    st = _lib.load().holo_bin_amplitudes(pa, a.numel() // (n * n), n, b,
                                         _ptr(out, torch.float32, None, "out"),
                                         ctypes.c_void_p(s.cuda_stream))
    _check(_lib.load(), None, st, "holo_bin_amplitudes")
    return out


def upsample2(x, stream=None):
    """Complex fields [..., n, n] (complex64 CUDA) extrapolated to [..., 2n, 2n] by linear
    interpolation at the fine pixel centres (holo_upsample2)."""
    import torch
    n = x.shape[-1]
    if x.shape[-2] != n:
        raise ValueError("square images")
    out = torch.empty(x.shape[:-2] + (2 * n, 2 * n), dtype=torch.complex64, device=x.device)
    px = _ptr(x, torch.complex64, None, "x")
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    st = _lib.load().holo_upsample2(px, x.numel() // (n * n), n,
                                    _ptr(out, torch.complex64, None, "out"),
                                    ctypes.c_void_p(s.cuda_stream))
    _check(_lib.load(), None, st, "holo_upsample2")
    return out


class Holo:
    """One reconstruction problem's geometry and workspace on one GPU.

    n: psi/detector side; pad: P (0 -> 2n); n_angles, n_dist: N_theta, N_z; chunk: angles
    per evaluation; wavelength, pixel, Z [m]; z: focus-to-sample distances [m];
    w_ref: weight of the reference-image term; ext: free-space value of the resample.
    """

    def __init__(self, n, n_angles, n_dist, wavelength, pixel, Z, z, pad=0, chunk=0,
                 w_ref=1.0, ext=1.0, stream=None):
        import torch
        self.lib = _lib.load()
        if len(z) != n_dist or n_dist > _lib.MAX_DIST:
            raise ValueError("len(z) must equal n_dist <= 8")
        g = _lib.HoloGeometry()
        g.n, g.pad, g.n_angles, g.n_dist, g.chunk = n, pad, n_angles, n_dist, chunk
        g.wavelength, g.pixel, g.Z = wavelength, pixel, Z
        for j, zj in enumerate(z):
            g.z[j] = zj
        g.w_ref, g.ext = w_ref, ext
        self.geometry = g
        self.n, self.P = n, (pad or 2 * n)
        self.n_angles, self.n_dist = n_angles, n_dist
        self.chunk = chunk or n_angles
        self.device = torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        handle = ctypes.c_void_p()
        st = self.lib.holo_create(ctypes.byref(g), ctypes.c_void_p(stream.cuda_stream),
                                  ctypes.byref(handle))
        _check(self.lib, None, st, "holo_create")
        self.ctx = handle
        self._keep = {}
        self.functional = "amplitude"

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.holo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- set-up
    def set_shifts(self, t):
        """t_kj (y, x) in pixels: float32 [n_angles][n_dist][2] (numpy, host)."""
        t = np.ascontiguousarray(t, dtype=np.float32)
        p = _host_ptr(t, np.float32, (self.n_angles, self.n_dist, 2), "shifts")
        _check(self.lib, self.ctx, self.lib.holo_set_shifts(self.ctx, p), "holo_set_shifts")

    def set_probe_shifts(self, s):
        """Probe shifts s_kj (y, x) in pixels: float32 [n_angles][n_dist][2] (numpy, host), or
        None to clear them (holo_set_probe_shifts)."""
        if s is None:
            p = ctypes.c_void_p(None)
        else:
            s = np.ascontiguousarray(s, dtype=np.float32)
            p = _host_ptr(s, np.float32, (self.n_angles, self.n_dist, 2), "probe shifts")
        _check(self.lib, self.ctx, self.lib.holo_set_probe_shifts(self.ctx, p),
               "holo_set_probe_shifts")

    def set_data(self, sqrt_d, sqrt_dref=None):
        """sqrt(d~_kj): float32 cuda [n_angles][n_dist][n][n]; sqrt(d~^r): [n][n] or None."""
        import torch
        n = self.n
        pd = ctypes.c_void_p(None)
        if sqrt_d is not None:
            pd = _ptr(sqrt_d, torch.float32, (self.n_angles, self.n_dist, n, n), "sqrt_d")
        pr = ctypes.c_void_p(None)
        if sqrt_dref is not None:
            pr = _ptr(sqrt_dref, torch.float32, (n, n), "sqrt_dref")
        _check(self.lib, self.ctx, self.lib.holo_set_data(self.ctx, pd, pr), "holo_set_data")
        # the amplitudes are copied by the library; the reference image is used in place
        self._keep["data"] = sqrt_dref

    def set_probe(self, q):
        """q: complex64 cuda [P][P]; computes p_j = D_{omega_j} q and C D_{zeta_0} q."""
        import torch
        p = _ptr(q, torch.complex64, (self.P, self.P), "q")
        _check(self.lib, self.ctx, self.lib.holo_set_probe(self.ctx, p), "holo_set_probe")

    # ---------------------------------------------------------------- evaluations
    def forward(self, psi, k0=0, u_out=None):
        """F2 over angles [k0, k0 + len(psi)); optionally the fields u_kj into u_out."""
        import torch
        nk = psi.shape[0]
        pp = _ptr(psi, torch.complex64, (nk, self.n, self.n), "psi")
        pu = ctypes.c_void_p(None)
        if u_out is not None:
            pu = _ptr(u_out, torch.complex64, (nk, self.n_dist, self.n, self.n), "u_out")
        loss = ctypes.c_double(0.0)
        st = self.lib.holo_forward(self.ctx, k0, nk, pp, pu, ctypes.byref(loss))
        _check(self.lib, self.ctx, st, "holo_forward")
        return loss.value

    def gradient(self, psi, grad_psi=None, grad_q=None, k0=0, accumulate=False, loss_in=0.0,
                 want_loss=True, accumulate_q=False, defer_q=False):
        """(F2, grad_psi, grad_q) over angles [k0, k0 + len(psi)) (Eq. gradpsi).

        accumulate: add to grad_psi, grad_q and loss_in; accumulate_q: add to grad_q and
        loss_in only (the chunks of one problem own disjoint psi slices but share q);
        defer_q: keep the probe-gradient sources for finish_q instead (grad_q is returned as
        None)."""
        import torch
        nk = psi.shape[0]
        pp = _ptr(psi, torch.complex64, (nk, self.n, self.n), "psi")
        if grad_psi is None:
            grad_psi = torch.empty_like(psi)
        if grad_q is None and not defer_q:
            grad_q = torch.empty((self.P, self.P), dtype=torch.complex64, device=psi.device)
        pg = _ptr(grad_psi, torch.complex64, (nk, self.n, self.n), "grad_psi")
        pq = ctypes.c_void_p(None) if defer_q else _ptr(grad_q, torch.complex64, (self.P, self.P),
                                                        "grad_q")
        loss = ctypes.c_double(loss_in)
        lp = ctypes.byref(loss) if want_loss else None
        flags = ((_lib.ACCUMULATE if accumulate else 0) | (_lib.ACCUMULATE_Q if accumulate_q else 0)
                 | (_lib.DEFER_Q if defer_q else 0))
        st = self.lib.holo_gradient(self.ctx, k0, nk, pp, lp, pg, pq, flags)
        _check(self.lib, self.ctx, st, "holo_gradient")
        return (loss.value if want_loss else None), grad_psi, (None if defer_q else grad_q)

    def finish_q(self, grad_q=None, accumulate=False):
        """holo_finish_q: grad_q (written, or added to) from the deferred sources."""
        import torch
        if grad_q is None:
            grad_q = torch.empty((self.P, self.P), dtype=torch.complex64, device=self.device)
        pq = _ptr(grad_q, torch.complex64, (self.P, self.P), "grad_q")
        st = self.lib.holo_finish_q(self.ctx, pq, _lib.ACCUMULATE_Q if accumulate else 0)
        _check(self.lib, self.ctx, st, "holo_finish_q")
        return grad_q

    def gradient_host(self, psi, sqrt_d=None, q=None, k0=0, grad_psi=None, grad_q=None):
        """holo_gradient_host: numpy in, numpy out (host buffers; copies inside the call)."""
        nk = psi.shape[0]
        n, P = self.n, self.P
        pp = _host_ptr(psi, np.complex64, (nk, n, n), "psi")
        pd = ctypes.c_void_p(None)
        if sqrt_d is not None:
            pd = _host_ptr(sqrt_d, np.float32, (nk, self.n_dist, n, n), "sqrt_d")
        pq = ctypes.c_void_p(None)
        if q is not None:
            pq = _host_ptr(q, np.complex64, (P, P), "q")
        if grad_psi is None:
            grad_psi = np.empty((nk, n, n), np.complex64)
        if grad_q is None:
            grad_q = np.empty((P, P), np.complex64)
        pg = _host_ptr(grad_psi, np.complex64, (nk, n, n), "grad_psi")
        pgq = _host_ptr(grad_q, np.complex64, (P, P), "grad_q")
        loss = ctypes.c_double(0.0)
        st = self.lib.holo_gradient_host(self.ctx, k0, nk, pp, pd, pq, ctypes.byref(loss), pg,
                                         pgq, 0)
        _check(self.lib, self.ctx, st, "holo_gradient_host")
        return loss.value, grad_psi, grad_q

    def propagate(self, x, z, out=None):
        """D_z of a P x P complex64 field (Appendix A, Eq. defGz)."""
        import torch
        px = _ptr(x, torch.complex64, (self.P, self.P), "x")
        if out is None:
            out = torch.empty_like(x)
        po = _ptr(out, torch.complex64, (self.P, self.P), "out")
        st = self.lib.holo_propagate(self.ctx, px, po, ctypes.c_double(z))
        _check(self.lib, self.ctx, st, "holo_propagate")
        return out

    # ---------------------------------------------------------------- CG vector ops
    def dot(self, a, b):
        """Re <a, b> in FP64 (Eq. DaiYuan2 inner products)."""
        import torch
        if a.shape != b.shape:
            raise ValueError("shape mismatch")
        pa = _ptr(a, torch.complex64, None, "a")
        pb = _ptr(b, torch.complex64, None, "b")
        out = ctypes.c_double(0.0)
        st = self.lib.holo_dot(self.ctx, pa, pb, a.numel(), ctypes.byref(out))
        _check(self.lib, self.ctx, st, "holo_dot")
        return out.value

    def step(self, x, eta, gamma):
        """x += gamma * eta."""
        import torch
        if x.shape != eta.shape:
            raise ValueError("shape mismatch")
        st = self.lib.holo_step(self.ctx, _ptr(x, torch.complex64, None, "x"),
                                _ptr(eta, torch.complex64, None, "eta"), float(gamma), x.numel())
        _check(self.lib, self.ctx, st, "holo_step")

    def direction(self, eta, g, beta):
        """eta = -g + beta * eta (Eq. DaiYuan2)."""
        import torch
        if eta.shape != g.shape:
            raise ValueError("shape mismatch")
        st = self.lib.holo_direction(self.ctx, _ptr(eta, torch.complex64, None, "eta"),
                                     _ptr(g, torch.complex64, None, "g"), float(beta), eta.numel())
        _check(self.lib, self.ctx, st, "holo_direction")

    def initial_probe(self, sqrt_dref, out=None):
        """q0 = D_{-zeta_0} of the reference amplitude embedded with repeated edges (the
        paper's initial probe: the reference image propagated back to sample plane 0)."""
        import torch
        pa = _ptr(sqrt_dref, torch.float32, (self.n, self.n), "sqrt_dref")
        if out is None:
            out = torch.empty((self.P, self.P), dtype=torch.complex64, device=self.device)
        po = _ptr(out, torch.complex64, (self.P, self.P), "out")
        _check(self.lib, self.ctx, self.lib.holo_initial_probe(self.ctx, pa, po),
               "holo_initial_probe")
        return out

    def set_functional(self, which):
        """'amplitude' (F2, Eq. min1; data are amplitudes) or 'intensity' (F1, Eq. min2; data
        are intensities) for the evaluations that follow."""
        code = {"amplitude": _lib.F2_AMPLITUDE, "intensity": _lib.F1_INTENSITY}[which]
        _check(self.lib, self.ctx, self.lib.holo_set_functional(self.ctx, code),
               "holo_set_functional")
        self.functional = which

    def dy_dots(self, g, g_prev, eta):
        """(Re <g, g>, Re <g, eta>, Re <g_prev, eta>) in one pass (Eq. DaiYuan2)."""
        import torch
        if not (g.shape == g_prev.shape == eta.shape):
            raise ValueError("shape mismatch")
        out = (ctypes.c_double * 3)()
        st = self.lib.holo_dy_dots(self.ctx, _ptr(g, torch.complex64, None, "g"),
                                   _ptr(g_prev, torch.complex64, None, "g_prev"),
                                   _ptr(eta, torch.complex64, None, "eta"), g.numel(), out)
        _check(self.lib, self.ctx, st, "holo_dy_dots")
        return out[0], out[1], out[2]

    def direction_step(self, x, eta, g, beta, gamma, dy=False):
        """eta = -g + beta * eta, then x += gamma * eta, in one pass.  dy: also form
        Re <g, eta_new> (holo_direction_step_dy; read_dy()[2])."""
        import torch
        if not (x.shape == eta.shape == g.shape):
            raise ValueError("shape mismatch")
        fn = self.lib.holo_direction_step_dy if dy else self.lib.holo_direction_step
        st = fn(self.ctx, _ptr(x, torch.complex64, None, "x"),
                _ptr(eta, torch.complex64, None, "eta"), _ptr(g, torch.complex64, None, "g"),
                float(beta), float(gamma), x.numel())
        _check(self.lib, self.ctx, st, "holo_direction_step_dy" if dy else "holo_direction_step")

    def set_dy_direction(self, eta):
        """holo_set_dy_direction: while set (a complex64 CUDA tensor laid out as grad_psi of
        the following gradient calls; None clears it), gradient() also forms Re <g, g> and
        Re <g, eta> of the grad_psi it writes (read_dy()[0:2])."""
        import torch
        p = ctypes.c_void_p(None)
        if eta is not None:
            p = _ptr(eta, torch.complex64, None, "eta")
        _check(self.lib, self.ctx, self.lib.holo_set_dy_direction(self.ctx, p),
               "holo_set_dy_direction")
        self._keep["dy"] = eta

    def read_dy(self):
        """holo_read_dy: (Re <g, g>, Re <g, eta>) of the last gradient with a direction set and
        Re <g, eta_new> of the last direction_step(..., dy=True); beta_DY = a / (b - c)."""
        out = (ctypes.c_double * 3)()
        _check(self.lib, self.ctx, self.lib.holo_read_dy(self.ctx, out), "holo_read_dy")
        return out[0], out[1], out[2]

    def set_stream(self, stream):
        """Issue later work on `stream` (a torch.cuda.Stream)."""
        _check(self.lib, self.ctx, self.lib.holo_set_stream(self.ctx, ctypes.c_void_p(stream.cuda_stream)),
               "holo_set_stream")
        self.stream = stream

    def read_loss(self):
        """F2 of the last evaluation (synchronises the context's stream)."""
        out = ctypes.c_double(0.0)
        _check(self.lib, self.ctx, self.lib.holo_read_loss(self.ctx, ctypes.byref(out)),
               "holo_read_loss")
        return out.value

    def set_timing(self, enable=True):
        """Start (and clear) or stop per-pass CUDA-event timing on the context's stream."""
        _check(self.lib, self.ctx, self.lib.holo_set_timing(self.ctx, 1 if enable else 0),
               "holo_set_timing")

    def get_timing(self):
        """{pass: (ms, launches)} summed since set_timing(True)."""
        ms = (ctypes.c_double * len(_lib.TIMERS))()
        nl = (ctypes.c_longlong * len(_lib.TIMERS))()
        _check(self.lib, self.ctx, self.lib.holo_get_timing(self.ctx, ms, nl), "holo_get_timing")
        return {name: (ms[i], nl[i]) for i, name in enumerate(_lib.TIMERS)}

    def set_schedule(self, row_blocks_per_sm=0, pass_b_stage=-1, pass_b_split=-1):
        """holo_set_schedule: resident row-pass blocks per SM (0: as many as fit), pass B's
        TMA stage (-1 auto, 0 off) and the split of its partial last round of column groups
        (-1 auto, 0 never, 1 plane-split kernel, 2 inside the staged kernel)."""
        st = self.lib.holo_set_schedule(self.ctx, row_blocks_per_sm, pass_b_stage, pass_b_split)
        _check(self.lib, self.ctx, st, "holo_set_schedule")
        self.schedule = (row_blocks_per_sm, pass_b_stage, pass_b_split)

    def set_device_error(self, word=1):
        """Test hook (holo_set_device_error): set the device error word as if a bounded
        device wait had given up (word 1; the next loss read raises HOLO_ERR_TIMEOUT) or a
        device bounds check had failed (bit 2: HOLO_ERR_BOUNDS); the read clears it."""
        st = self.lib.holo_set_device_error(self.ctx, ctypes.c_ulonglong(word))
        _check(self.lib, self.ctx, st, "holo_set_device_error")

    def workspace_bytes(self):
        v = ctypes.c_longlong(0)
        _check(self.lib, self.ctx, self.lib.holo_workspace_bytes(self.ctx, ctypes.byref(v)),
               "holo_workspace_bytes")
        return v.value

    def launch_count(self):
        v = ctypes.c_longlong(0)
        _check(self.lib, self.ctx, self.lib.holo_launch_count(self.ctx, ctypes.byref(v)),
               "holo_launch_count")
        return v.value
