/*
 * holo.h - C ABI of the GB300 holography functional library.
 *
 * The library evaluates, on one GPU, the multi-distance cone-beam holography functional
 * with simultaneous probe retrieval of Nikitin et al., "X-ray nano-holotomography
 * reconstruction with simultaneous probe retrieval" (Sec. 2), and its gradients:
 *
 *   u_kj  = L_kj(psi_k) = C D_{zeta_j/m~_j^2}( D_{omega_j}(S_{s_kj} q) * M_{1/m~_j}(S_{t_kj} psi_k) )
 *                                                   (Eq. fwd_model_cone3 with the shifts of Eq. min1;
 *                                                    probe shifts s_kj are zero unless
 *                                                    holo_set_probe_shifts sets them)
 *   F2    = sum_kj || |u_kj| - sqrt(d~_kj) ||^2 + w_ref || |C D_{zeta_0} q| - sqrt(d~^r) ||^2
 *                                                   (Eq. min1)
 *   grad_psi_k F2 = 2 sum_j L*_kj( u - sqrt(d~) u/|u| )        (Eq. gradpsi)
 *   grad_q F2     = 2 ( sum_kj Q*_kj(...) + D*_{zeta_0}(...) ) (probe gradient after Eq. gradpsi)
 *
 * with m~_j = z_j/z_0, omega_j = (z_j - z_0)/m~_j, zeta_j = z_j (Z - z_j)/Z (Sec. 2;
 * Theorem t3 of Appendix A), D_z Fresnel propagation (Appendix A, Eq. defPz/defGz), M the
 * dilation and S the lateral shift.  Discretisation (the paper gives none):
 *   - psi_k is n x n; q and all propagations live on a P x P grid (P = 2n by default);
 *     the detector is the central n x n crop C of the P x P grid.
 *   - D_z multiplies the DFT of the P x P field by exp(-i pi lambda z (fx^2 + fy^2)),
 *     f = k/(P pixel), k in [-P/2, P/2).
 *   - M_{1/m~} S_t psi is bilinear interpolation of psi at psi-coordinate m~ x - t
 *     (pixels; pixel centres at i - n/2 for psi and i - P/2 for the P x P grid), with
 *     the value `ext` outside psi's n x n domain.  Gradients use its exact transpose.
 *   - Gradients are real gradients for <a, b> = Re sum conj(a) b: dF(x; h) = Re <grad, h>.
 *
 * Conventions for every entry point:
 *   - Complex arrays are interleaved complex64 (float re, float im), row-major, densely
 *     packed.  "dev" pointers are CUDA device pointers on the context's device; "host"
 *     pointers are CPU memory (pinned memory makes copies faster).
 *   - The caller owns every array it passes; the library never frees them.  Device
 *     arrays registered with holo_set_data must stay valid until the next holo_set_data
 *     or holo_destroy.  The context owns only its workspace (probe planes, tables,
 *     per-plane intermediates, partial sums).
 *   - Work is issued on the stream given to holo_create.  Calls that return a host
 *     scalar (loss, inner product) synchronise that stream before returning; all other
 *     calls are asynchronous with respect to the host.
 *   - Every entry point returns a holo_status and never aborts the process.  Invalid
 *     arguments are rejected before any device work (HOLO_ERR_ARG); CUDA failures return
 *     HOLO_ERR_CUDA (details in holo_last_error).  Calls in the wrong order (e.g. a
 *     gradient before holo_set_probe) return HOLO_ERR_STATE.
 *   - Device waits are bounded.  Where the column pass stages its input tiles by TMA
 *     (P >= 1024, even n), a tile that does not arrive within the bound makes the kernel
 *     return early and set a device error word; the next call that reads a loss (any call
 *     returning a loss, holo_read_loss) returns HOLO_ERR_TIMEOUT, clears the word, and the
 *     results of the evaluations since the previous loss read are invalid.
 *   - A library built with HOLO_BOUNDS_CHECK defined (paper_2407_20304_gb300/build.py,
 *     bounds_check=True: _build_bc/libholo.so) also checks its table-driven device indices
 *     (line-table entries, plane boxes against the workspace strides, transposed taps); a
 *     failed check skips the access and sets bit 2 of the same word, and the next loss read
 *     returns HOLO_ERR_BOUNDS (before HOLO_ERR_TIMEOUT when both are set).  Nothing traps.
 */
#ifndef HOLO_H
#define HOLO_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct holo_ctx holo_ctx;

typedef enum {
  HOLO_OK = 0,
  HOLO_ERR_ARG = 1,         /* invalid argument (null pointer, bad size, bad geometry) */
  HOLO_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
  HOLO_ERR_OOM = 3,         /* workspace allocation failed */
  HOLO_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
  HOLO_ERR_STATE = 5,       /* call order: shifts / data / probe not set yet */
  HOLO_ERR_NUMERIC = 6,     /* non-finite loss */
  HOLO_ERR_UNSUPPORTED = 7, /* valid but unsupported size (e.g. P = 80 or P > 4096) */
  HOLO_ERR_BOUNDS = 8       /* a device bounds check failed (HOLO_BOUNDS_CHECK builds only) */
} holo_status;

#define HOLO_MAX_DIST 8

/* Functionals (holo_set_functional). */
#define HOLO_F2_AMPLITUDE 0 /* F2 of Eq. min1: data are amplitudes sqrt(d~) (the default) */
#define HOLO_F1_INTENSITY 1 /* F1 of Eq. min2: data are intensities d~ */

/* Flags of holo_gradient / holo_gradient_host. */
#define HOLO_ACCUMULATE 1u   /* add to grad_psi, grad_q and *loss instead of overwriting */
#define HOLO_ACCUMULATE_Q 2u /* add to grad_q and *loss only; grad_psi is overwritten (chunks
                                of one problem own disjoint psi slices but share q) */
#define HOLO_DEFER_Q 4u      /* holo_gradient: keep the chunk's probe-gradient sources in the
                                context instead of propagating them into grad_q (see
                                holo_finish_q); grad_q may be NULL */

/*
 * Instrument geometry and discretisation (Table 1 lists the paper's instrument).
 *   n           psi / detector side in pixels; even, 16 <= n <= pad.
 *   pad         P, the side of the grid on which q lives and fields propagate; 0 means
 *               2n.  Supported: 2^k (16 .. 4096) and 3 * 2^k (48 .. 3072), with
 *               P - n even.
 *   n_angles    N_theta: number of projection angles of the whole problem (indexing of
 *               shifts and data).
 *   n_dist      N_z: number of sample planes, 1 .. HOLO_MAX_DIST.
 *   chunk       maximum angles per forward / gradient call (workspace size); 0 means
 *               n_angles.
 *   wavelength  lambda [m]; pixel: object-plane pixel size [m] (detector pixel / m0);
 *   Z           focus-to-detector distance [m]; z[j]: focus-to-sample distances [m],
 *               0 < z[0] < z[1] < ... < Z.
 *   w_ref       weight of the reference-image term of Eq. min1 (0 disables it).
 *   ext         free-space value of the resample: 1 (transmittance of empty space) or 0
 *               (a test mode in which the model is bilinear in (psi, q)).
 */
typedef struct {
  int n;
  int pad;
  int n_angles;
  int n_dist;
  int chunk;
  double wavelength;
  double pixel;
  double Z;
  double z[HOLO_MAX_DIST];
  double w_ref;
  double ext;
} holo_geometry;

/* Create a context on the current CUDA device.  `stream` is a cudaStream_t (NULL: the
 * legacy default stream).  Derives m~_j, omega_j, zeta_j (Sec. 2) and builds the FP64
 * chirp and twiddle tables.  On failure *out is set to NULL. */
holo_status holo_create(const holo_geometry* geo, void* stream, holo_ctx** out);

/* Free the context's workspace.  NULL is accepted. */
holo_status holo_destroy(holo_ctx* ctx);

/* Sample shifts t_kj of Eq. min1 (S_{t_kj} psi_k), host float [n_angles][n_dist][2] as
 * (t_y, t_x) in psi pixels, copied.  Sizes the per-plane workspace; must precede
 * holo_forward / holo_gradient.  Probe shifts s_kj are zero unless
 * holo_set_probe_shifts sets them. */
holo_status holo_set_shifts(holo_ctx* ctx, const float* t_host);

/* Probe shifts s_kj of Eq. min1 / Eq. min2 (the S_{s_kj} q inside D_{omega_j}), host float
 * [n_angles][n_dist][2] as (s_y, s_x) in pixels of the padded grid, copied; NULL clears
 * them.  |s| <= n/2 per component, else HOLO_ERR_ARG.  The shift is moved off the probe as
 * Sec. 2 remarks after Eq. min2 (shifts commute with the other operators), so q is never
 * interpolated:
 *   u_kj = C S_s D_{zhat_j}( p_j * M_{1/m~_j} S_{t_kj - m~_j s_kj} psi_k ),
 * with S_s the band-limited shift (phase ramp exp(-2 pi i k s / P) on the DFT, k in
 * [-P/2, P/2)); for integer s this is exactly Eq. min1 with q rolled by s.  The ext-part of
 * every plane then moves with s, so the per-plane box becomes the whole P x P grid: more
 * row transforms per plane and a per-plane workspace of P x n + P x P complex64 per plane
 * slot.  May be called before or after holo_set_shifts (the planes are rebuilt). */
holo_status holo_set_probe_shifts(holo_ctx* ctx, const float* s_host);

/* Register the data: sqrt_d (dev float [n_angles][n_dist][n][n]) holds sqrt(d~_kj), the
 * amplitudes of the data rescaled to the plane-0 grid (d~ = m0^2 M_{1/m0} d, Sec. 2);
 * sqrt_dref (dev float [n][n], may be NULL when w_ref = 0) holds sqrt(d~^r).  sqrt_d is
 * copied into the workspace (in the column-blocked layout the column pass reads: the columns
 * of one column group contiguous per row) and the stream is synchronised, so the caller may
 * reuse or free it when the call returns; sqrt_dref is not copied and must stay valid while
 * used.  sqrt_d may be NULL when every evaluation passes its chunk's data through
 * holo_gradient_host (only the reference is kept). */
holo_status holo_set_data(holo_ctx* ctx, const float* sqrt_d, const float* sqrt_dref);

/* Set the probe q (dev complex64 [P][P]) and compute its propagations p_j = D_{omega_j} q
 * (Eq. fwd_model_cone3) and the reference field C D_{zeta_0} q (copied into the
 * workspace; q itself is not retained). */
holo_status holo_set_probe(holo_ctx* ctx, const void* q);

/* Forward model and F2 restricted to angles [k0, k0 + nk) (Eq. fwd_model_cone3,
 * Eq. min1).  psi: dev complex64 [nk][n][n].  u_out: dev complex64 [nk][n_dist][n][n]
 * receiving u_kj, or NULL.  loss (host, may be NULL): sum over the chunk's planes of
 * || |u| - sqrt(d~) ||^2, plus the reference term when k0 == 0.  Requires 1 <= nk <=
 * chunk and k0 + nk <= n_angles. */
holo_status holo_forward(holo_ctx* ctx, int k0, int nk, const void* psi, void* u_out,
                         double* loss);

/* F2 and its gradients over angles [k0, k0 + nk) (Eq. gradpsi and the probe gradient
 * after it).  psi: dev complex64 [nk][n][n]; grad_psi: dev complex64 [nk][n][n];
 * grad_q: dev complex64 [P][P] (the chunk's contribution; the reference term is included
 * when k0 == 0).  loss: host, may be NULL.  flags: HOLO_ACCUMULATE adds to grad_psi,
 * grad_q and *loss; HOLO_ACCUMULATE_Q adds to grad_q and *loss only (summing the chunks of
 * one problem); otherwise all are overwritten. */
holo_status holo_gradient(holo_ctx* ctx, int k0, int nk, const void* psi, double* loss,
                          void* grad_psi, void* grad_q, unsigned flags);

/* Deferred probe gradient.  grad_q is linear in two sources per chunk: the residual sum
 * T = ext sum_kj r_kj + w_ref r_ref and, per distance j, G'_j = sum_k conj(w_kj) v_kj; each
 * chunk's share is propagated by J + 1 P x P Fresnel steps.  A gradient call with
 * HOLO_DEFER_Q instead adds its sources to the context's accumulators (held on the union of
 * every plane's box of distance j), starting them afresh unless HOLO_ACCUMULATE or
 * HOLO_ACCUMULATE_Q is set, and leaves grad_q alone; holo_finish_q then writes (or with
 * HOLO_ACCUMULATE_Q adds) grad_q = 2 [D_{-zeta_0}(C* T) + sum_j D_{-omega_j}(G'_j)] once for
 * all the deferred chunks.  The loss and grad_psi are not deferred.  A gradient call without
 * HOLO_DEFER_Q discards pending sources; holo_finish_q without pending sources returns
 * HOLO_ERR_STATE.  The accumulators (about J (n + 16)^2 complex64) are allocated by the first
 * deferred call.  Summing the sources before propagating rounds differently from summing the
 * propagated chunks (equal to rounding).  holo_gradient_host does not take HOLO_DEFER_Q. */
holo_status holo_finish_q(holo_ctx* ctx, void* grad_q, unsigned flags);

/* holo_gradient with host buffers: copies psi_host ([nk][n][n]) and, when not NULL,
 * sqrt_d_host (float [nk][n_dist][n][n], the chunk's data, used instead of the data
 * registered with holo_set_data) and q_host ([P][P], then holo_set_probe) to the
 * device, evaluates, and copies grad_psi_host ([nk][n][n]) and grad_q_host ([P][P])
 * back.  HOLO_ACCUMULATE applies to *loss only.  Staging buffers are allocated on the
 * first call and kept. */
holo_status holo_gradient_host(holo_ctx* ctx, int k0, int nk, const void* psi_host,
                               const float* sqrt_d_host, const void* q_host, double* loss,
                               void* grad_psi_host, void* grad_q_host, unsigned flags);

/* Fresnel propagation D_z of a P x P field (Appendix A, Eq. defGz): out = D_z(in),
 * dev complex64 [P][P] each (in == out allowed). */
holo_status holo_propagate(holo_ctx* ctx, const void* in, void* out, double z);

/* Re <a, b> = Re sum conj(a_i) b_i over n_c64 complex64 elements (dev), accumulated in
 * FP64: the inner products of the Dai-Yuan coefficient (Eq. DaiYuan2) and the step
 * length. */
holo_status holo_dot(holo_ctx* ctx, const void* a, const void* b, long long n_c64,
                     double* re_out);

/* x += gamma * eta over n_c64 complex64 elements (dev): the CG update
 * psi^(m+1) = psi^(m) + gamma eta (Sec. 2). */
holo_status holo_step(holo_ctx* ctx, void* x, const void* eta, double gamma, long long n_c64);

/* eta = -g + beta * eta over n_c64 complex64 elements (dev): the conjugate direction of
 * Eq. DaiYuan2 (beta = 0 restarts with the steepest-descent direction). */
holo_status holo_direction(holo_ctx* ctx, void* eta, const void* g, double beta,
                           long long n_c64);

/* Hierarchical reconstruction (Sec. 3, on speeding up: iterations on binned data, then the
 * recovered object and probe extrapolated to a grid twice as dense).  Context-free,
 * asynchronous on `stream` (a cudaStream_t, NULL for the legacy stream).
 * holo_bin_amplitudes: count amplitude images (dev f32 [count][n][n]) -> binned amplitudes
 *   (dev f32 [count][n/b][n/b]) = sqrt(mean of a^2 over b x b blocks), i.e. the intensities
 *   are averaged.  HOLO_ERR_ARG unless n is a multiple of b >= 1.
 * holo_upsample2: count complex images (dev complex64 [count][n][n]) -> [count][2n][2n] by
 *   linear interpolation at the fine pixel centres (fine pixel f at coarse coordinate
 *   (f + 1/2)/2 - 1/2), edges clamped.  in and out must not overlap. */
holo_status holo_bin_amplitudes(const float* in, long long count, int n, int b, float* out,
                                void* stream);
holo_status holo_upsample2(const void* in, long long count, int n, void* out, void* stream);

/* Initial probe (Sec. 2, on the initial guess): the reference image propagated back to
 * sample plane 0, q_out = D_{-zeta_0}(E sqrt_dref), where E embeds the n x n amplitude
 * sqrt_dref (dev f32 [n][n]) in the P x P grid by repeating its edge values.  q_out: dev
 * complex64 [P][P], caller-owned.  Asynchronous on the context's stream. */
holo_status holo_initial_probe(holo_ctx* ctx, const float* sqrt_dref, void* q_out);

/* Select the functional that holo_forward / holo_gradient(_host) evaluate from now on:
 * HOLO_F2_AMPLITUDE (Eq. min1, |u| against the amplitudes sqrt(d~), the default) or
 * HOLO_F1_INTENSITY (Eq. min2, |u|^2 against the intensities d~; the reference term likewise,
 * weighted by w_ref).  The data registered with holo_set_data (and passed to
 * holo_gradient_host) are read as amplitudes or intensities accordingly.  F1's gradients use
 * r = 2 (|u|^2 - d~) u in place of r = u - sqrt(d~) u/|u|.  HOLO_ERR_ARG for other values. */
holo_status holo_set_functional(holo_ctx* ctx, int functional);

/* The three inner products of the Dai-Yuan coefficient (Eq. DaiYuan2) in one pass over
 * the vectors (dev complex64 [n_c64] each): out[0] = Re <g, g>, out[1] = Re <g, eta>,
 * out[2] = Re <g_prev, eta>, each accumulated like holo_dot (FP32 over 16 elements, then
 * FP64), so beta_DY = out[0] / (out[1] - out[2]).  out: host double[3], written before the
 * call returns (the context's stream is synchronised). */
holo_status holo_dy_dots(holo_ctx* ctx, const void* g, const void* g_prev, const void* eta,
                         long long n_c64, double* out);

/* eta = -g + beta * eta, then x += gamma * eta with the new eta, in one pass over the
 * vectors (dev complex64 [n_c64] each): holo_direction followed by holo_step, bit for bit. */
holo_status holo_direction_step(holo_ctx* ctx, void* x, void* eta, const void* g, double beta,
                                double gamma, long long n_c64);

/* The Dai-Yuan inner products (Eq. DaiYuan2) of the object part formed where the vectors
 * already stream through the GPU, so that a CG step needs no separate pass over them:
 * holo_set_dy_direction(ctx, eta): eta = dev complex64 laid out as the grad_psi of the
 *   following holo_gradient calls ([nk][n][n], 16-byte aligned; HOLO_ERR_ARG otherwise), or
 *   NULL to stop.  While it is set, every holo_gradient also forms Re <g, g> and Re <g, eta>
 *   of the grad_psi g it writes (after the HOLO_ACCUMULATE addition): FP32 over the
 *   elements of a psi row that one warp of 32 threads writes (n / 8 at most), then FP64
 *   across warps and rows.  The caller keeps
 *   eta alive while it is set; holo_gradient_host does not form the products.
 * holo_direction_step_dy: holo_direction_step that also forms Re <g, eta_new> with its new
 *   direction (accumulated like holo_dot).
 * holo_read_dy(ctx, out): synchronises the stream; out[0] = Re <g, g> and out[1] =
 *   Re <g, eta> of the last holo_gradient with a direction set, out[2] = Re <g, eta> of the
 *   last holo_direction_step_dy.  With eta_k set during the evaluation of g_{k+1}, and out[2]
 *   from the step that made eta_k from g_k, beta_DY = out[0] / (out[1] - out[2]): the three
 *   holo_dy_dots products without a pass of their own. */
holo_status holo_set_dy_direction(holo_ctx* ctx, const void* eta);
holo_status holo_direction_step_dy(holo_ctx* ctx, void* x, void* eta, const void* g,
                                   double beta, double gamma, long long n_c64);
holo_status holo_read_dy(holo_ctx* ctx, double* out);

/* Per-pass device timing (CUDA events recorded on the context's stream around each
 * launch group).  Pass ids: */
#define HOLO_T_PROBE 0   /* holo_set_probe: p_j = D_{omega_j} q and C D_{zeta_0} q */
#define HOLO_T_PASS_A 1  /* resample x probe, row propagation of the box rows */
#define HOLO_T_PASS_B 2  /* column propagation, amplitude residual, column adjoint */
#define HOLO_T_PASS_C 3  /* row adjoint, conj(p) v, x-transpose, conj(w) v */
#define HOLO_T_PASS_D 4  /* y-transpose, sum over distances -> grad_psi */
#define HOLO_T_QGRAD 5   /* reductions and propagations of grad_q */
#define HOLO_T_REDUCE 6  /* FP64 loss / inner-product reductions */
#define HOLO_T_VECTOR 7  /* CG vector updates (step, direction) */
#define HOLO_NUM_TIMERS 8

/* enable != 0 starts recording (and clears earlier records); 0 stops. */
holo_status holo_set_timing(holo_ctx* ctx, int enable);

/* Synchronises the stream and returns, per pass id, the summed device time in ms and the
 * number of kernel launches recorded since holo_set_timing(ctx, 1).  Arrays of
 * HOLO_NUM_TIMERS entries; either may be NULL. */
holo_status holo_get_timing(holo_ctx* ctx, double* ms, long long* launches);

/* Re <a, b> like holo_dot, for callers that cannot allocate device memory: no context is
 * needed and nothing is allocated (the paper has no counterpart; this is an interface
 * for embedders).  a, b: dev complex64 [n_c64] on the CURRENT device (device or managed
 * memory; anything else, e.g. host memory or another device's memory, returns HOLO_ERR_ARG
 * before any device work); re_out: host, written after the call synchronises `stream` (a
 * cudaStream_t of the current device, NULL for the legacy default stream).  The per-block
 * partial sums live in a fixed 512 KiB device array inside the library (held on every GPU
 * that loads it until the process exits), so n_c64 may be at most 268435456 (2^28);
 * longer inputs return HOLO_ERR_UNSUPPORTED before any device work.  The first call on a
 * device looks up that array's device address (with the device current).  All calls share
 * the array: calls that overlap on the GPU race.
 * There is no context to hold error text: HOLO_ERR_CUDA comes without details. */
holo_status holo_dot_noalloc(const void* a, const void* b, long long n_c64, double* re_out,
                             void* stream);

/* Issue the context's later work on `stream` (a cudaStream_t, NULL for the legacy
 * default stream), e.g. to place independent reconstructions on different branches of a
 * captured CUDA graph.  The caller orders it against work already issued. */
holo_status holo_set_stream(holo_ctx* ctx, void* stream);

/* Schedule of the context's passes (an autotuner's knobs; results do not depend on the first
 * two, the third changes only the summation order of grad_q's residual sum and the loss):
 *   row_blocks_per_sm  resident blocks per SM of the row passes A and C (0: as many as fit);
 *   pass_b_stage       pass B's TMA staging of its input tiles: -1 where it fits (default),
 *                      0 off (plain loads), 1 same as -1;
 *   pass_b_split       pass B's last, partial round of column groups: -1 automatic (default:
 *                      split by planes with the plane-split kernel when there are fewer than
 *                      three full rounds), 0 never split (whole column groups per block), 1
 *                      split by the plane-split kernel (no TMA stage), 2 split inside the
 *                      staged kernel, whenever the last round is partial.
 * HOLO_ERR_ARG for values outside these ranges. */
holo_status holo_set_schedule(holo_ctx* ctx, int row_blocks_per_sm, int pass_b_stage,
                              int pass_b_split);

/* Batched evaluation of independent problems (Sec. 4: independent angle chunks; here problems
 * of uneven sizes on one GPU), each an existing context with shifts and data set.  One batch
 * gradient evaluates, for every problem, the probe propagation and F2, grad_psi and grad_q
 * over all its angles (in chunks of the context's chunk size, summed like holo_gradient with
 * HOLO_ACCUMULATE_Q).  Passes A-D of the chunks of all problems run as persistent launches
 * that walk device work lists of (problem, work item) entries, one launch per pass and line
 * length (pass D: one for all); the reductions and the grad_q propagations run per problem.
 * The probe gradient's sources are summed over a problem's chunks and propagated once (as
 * holo_gradient with HOLO_DEFER_Q and holo_finish_q).  Every problem's results equal bit for
 * bit those of its own holo_set_probe, holo_gradient (HOLO_DEFER_Q, HOLO_ACCUMULATE_Q after
 * the first chunk) and holo_finish_q calls with the same schedule (holo_batch_prepare sets
 * pass_b_split = 0 on every context: the batched column pass works on whole column groups).
 *   holo_batch_create   keeps the array of `count` contexts (not owned; they must outlive
 *                       the batch);
 *   holo_batch_set_problem  the device buffers of problem i: psi [n_angles][n][n], q [P][P]
 *                       (complex64, read), grad_psi [n_angles][n][n] and grad_q [P][P]
 *                       (written);
 *   holo_batch_prepare  builds and uploads the work lists (allocates; synchronous); again
 *                       after any set_problem, holo_set_schedule or holo_set_shifts;
 *   holo_batch_gradient issues one evaluation of every problem on `stream` (a cudaStream_t,
 *                       NULL: the legacy stream; every context is switched to it).  Nothing
 *                       is allocated and the host does not wait, so the call can be captured
 *                       into a CUDA graph.  Losses: holo_read_loss of each context afterwards.
 *                       HOLO_ERR_STATE before prepare.  A bounded wait that gives up sets
 *                       every problem's error word (reported by its next loss read).
 *   holo_batch_destroy  frees the work lists (NULL accepted). */
typedef struct holo_batch holo_batch;
holo_status holo_batch_create(holo_ctx* const* ctxs, int count, holo_batch** out);
holo_status holo_batch_set_problem(holo_batch* b, int i, const void* psi, const void* q,
                                   void* grad_psi, void* grad_q);
holo_status holo_batch_prepare(holo_batch* b);
holo_status holo_batch_gradient(holo_batch* b, void* stream);
holo_status holo_batch_destroy(holo_batch* b);

/* F2 accumulated on the device: the loss of the last forward / gradient evaluation
 * (including the reference term when it had k0 == 0), plus the earlier ones since the
 * last evaluation issued without HOLO_ACCUMULATE / HOLO_ACCUMULATE_Q.  Read after
 * synchronising the stream; for evaluations issued without a host loss pointer, e.g.
 * inside a captured CUDA graph. */
holo_status holo_read_loss(holo_ctx* ctx, double* loss);

/* Fault injection for tests (no counterpart in the paper; nothing faults on the GPU).
 * holo_set_device_error writes `word` into the context's device error word, the word a
 * bounded device wait sets when it gives up (see the conventions above), as if such a wait
 * had expired: the next call that reads a loss returns HOLO_ERR_TIMEOUT (HOLO_ERR_BOUNDS if
 * bit 2 is set, as a failed bounds check sets it) and clears it (word 0 clears it now).
 * Synchronises the context's stream.
 * The environment variable HOLO_FAULT (a comma-separated list, read at every check)
 * injects host-side failures: "alloc" fails every workspace allocation (HOLO_ERR_OOM, before
 * cudaMalloc), "arg" rejects every forward / gradient call (HOLO_ERR_ARG, before device
 * work), "nan" makes every loss read report a non-finite loss (HOLO_ERR_NUMERIC). */
holo_status holo_set_device_error(holo_ctx* ctx, unsigned long long word);

/* Bytes of device workspace currently held by the context. */
holo_status holo_workspace_bytes(const holo_ctx* ctx, long long* bytes);

/* Kernel launches issued by the context since creation (a counter for benchmarks). */
holo_status holo_launch_count(const holo_ctx* ctx, long long* count);

/* Static text for a status code. */
const char* holo_status_string(holo_status s);

/* Text of the last error recorded in ctx (never NULL; "" when none). */
const char* holo_last_error(const holo_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HOLO_H */
