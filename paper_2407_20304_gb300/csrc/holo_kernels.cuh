// Kernels of the per-plane hot path, templated on the line length P.
//
// Forward model of one (k, j) plane (Eq. fwd_model_cone3 with the shifts of Eq. min1):
//   u_kj = C D_{zhat_j}( p_j * R_kj psi_k ),  zhat_j = zeta_j / m~_j^2,  p_j = D_{omega_j} q.
// The resample is affine, R psi = ext + w with w = R0(psi - ext) supported on a box of
// about n/m~_j pixels per side, so by linearity
//   u_kj = ext * C D_{zhat_j}(p_j) + C D_{zhat_j}(p_j * w_kj) = ext * b + C D_{zhat_j}(p_j * w_kj)
// with b = C D_{zeta_0}(q) the same for every plane (Theorem t3: zhat_j + omega_j = zeta_0).
// Only the box rows need the row transforms, and only box columns of the adjoint field
// are needed for grad_psi and for the w-part of grad_q.  Per plane:
//   pass A (rows of the box): x = p_j * w, row FFT, chirp, row IFFT, keep the n
//           detector columns -> Y[box rows][n]
//   pass B (detector columns): column FFT, chirp, IFFT, keep the n detector rows,
//           u = ext b + (.), residual r = u - a u/|u| (Eq. gradpsi), loss partial,
//           r stored for the ext-part of grad_q, then the adjoint column transform
//           (conjugate chirp) on C* r, keep box rows -> V (in place of Y)
//   pass C (rows of the box): adjoint row transform -> v on the box columns;
//           z = conj(p_j) v, x-transpose of the bilinear resample -> h[box rows][n]
//           (in place of V); conj(w) v -> per-plane buffer for grad_q
//   pass D (psi rows, line-length independent): y-transpose, sum over j, times 2.
//
// All passes run persistent blocks (a grid that fills the GPU once) that load the FFT
// twiddles into shared memory once and then walk a flat list of work items.
//
// Probe shifts s_kj (Eq. min1) use the SHIFT forms of passes A, B and C.  The shift is moved
// off the probe, u_kj = C S_s D_{zhat_j}(p_j * R'_kj psi_k) with R' the resample at object
// shift t - m~_j s, and S_s D_{zhat_j} is one separable Fourier multiplier: the chirp times
// the per-plane phase ramps exp(-2 pi i k s / P) of each axis (ramp_x in the row passes,
// ramp_y in the column pass; conjugated in the adjoints).  The ext-part of the field is then
// shifted per plane as well, so the box is the whole P x P grid, w holds R' psi itself
// (ext added back in pass A) and pass B runs with ext = 0 (no b term, T = w_ref r_ref).

#pragma once

#include <type_traits>

#include "holo_fft.cuh"
#include "holo_internal.h"
#include "holo_tma.cuh"

namespace holo {

// Block shapes.  Row passes keep each line in its own threads (coalesced along rows);
// column passes interleave C columns within a warp so that one load instruction covers
// whole 32-byte sectors of C adjacent columns.  Line strides in shared memory are
// chosen so that every exchange phase is free of bank conflicts (checked by simulating
// the address patterns for all P).
// Shared memory of every line kernel: the twiddle roots, the half chirp table (P/2 + 1
// entries) and the exchange lines.
template <int P>
struct SmemHead {
  static constexpr int ROOTS = (Fft<P>::ROOTS + 1) & ~1;
  // half chirp table; padded (entry i at i + i/16) where the frequency layout makes lanes
  // read entries 16 apart (Fft<P>::HW), so those reads stay free of bank conflicts
  static constexpr int CHIRP = ((Fft<P>::HW ? spad_c(P / 2) : P / 2) + 2) & ~1;
  static constexpr int WORDS = ROOTS + CHIRP;
};

// Lines per row block: about 256 threads, whole warps.
__host__ __device__ constexpr int row_lines(int T, int g = 0) {
  return T >= 256 ? 1 : (g == 0 ? row_lines(T, 256 / T) : ((g * T) % 32 ? row_lines(T, g - 1) : g));
}

template <int P>
struct RowCfg {
  static constexpr int T = P / 16;
  static constexpr int G = row_lines(T);                // lines per block
  static constexpr int NT = G * T;
  static constexpr int LS = Fft<P>::SMEM + (P == 64 || P == 192 ? 1 : 0);
  static constexpr size_t SMEM_BYTES = (size_t)(SmemHead<P>::WORDS + G * LS) * sizeof(float2);
  // resident blocks per SM asked of ptxas: 3 where that measured faster (the row passes then
  // fit in 80-96 registers with at most ~100 bytes of spills), else 2
  static constexpr int MINB = P == 4096 || P == 2048 || P == 1024 || P == 768 ? 3 : 2;
};

template <int P>
struct ColCfg {
  static constexpr int T = P / 16;
  static constexpr int C =
      Fft<P>::R3 ? (T >= 192 ? 2 : (T >= 24 ? 4 : (T >= 12 ? 8 : (T >= 6 ? 16 : 32))))
                 : (T >= 256 ? 2 : (T >= 64 ? 4 : (P == 512 ? 16 : 256 / T)));
  static constexpr int NT = C * T;
  static constexpr int EXTRA =
      Fft<P>::R3 ? (P == 768 ? 4 : (P == 1536 ? 3 : (P == 96 || P == 192 || P == 384 ? 1 : 0)))
                 : (P >= 4096 ? 8 : (P == 2048 ? 4 : (P == 1024 ? 3 : (P == 16 ? 0 : 1))));
  static constexpr int LS = Fft<P>::SMEM + EXTRA;
  static constexpr size_t SMEM_BYTES = (size_t)(SmemHead<P>::WORDS + C * LS) * sizeof(float2);
  static constexpr size_t PASS_B_SMEM = SMEM_BYTES;
};

// Sum of per-thread FP64 values over the block; result valid in thread 0.
__device__ __forceinline__ double block_sum_f64(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += red[i];
  }
  return s;
}

// Builds with HOLO_BOUNDS_CHECK check their table-driven indices on the device: a bad entry
// sets bit 2 of the problem's error word (HOLO_ERR_BOUNDS at the next loss read) and the access
// is skipped; nothing traps.  Other builds compile the checks away.
#if defined(HOLO_BOUNDS_CHECK)
constexpr bool kBoundsCheck = true;
#else
constexpr bool kBoundsCheck = false;
#endif

__device__ __forceinline__ void flag_bounds(unsigned long long* err) { atomicOr(err, 2ull); }

// A plane's box inside the P x P grid and inside the workspace strides of its problem.
__device__ __forceinline__ bool plane_box_ok(const PassArgs& a, const PlaneDesc& d, int P) {
  return d.by0 >= 0 && d.bys >= 0 && d.by0 + d.bys <= P && d.bx0 >= 0 && d.bxs >= 0 &&
         d.bx0 + d.bxs <= P && d.bys <= a.tap_stride && d.bxs <= a.tap_stride &&
         (long long)d.bys * a.n <= a.ystride && (long long)d.bys * d.bxs <= a.gkstride;
}

// A row-pass line (plane gp, box row i): the plane among the chunk's, the row inside its box.
__device__ __forceinline__ bool line_ok(const PassArgs& a, int gp, int i, int P) {
  const int p_lo = a.k0 * a.J;
  if (gp < p_lo || gp >= p_lo + a.nk * a.J) return false;
  const PlaneDesc d = a.planes[gp];
  return i >= 0 && i < d.bys && plane_box_ok(a, d, P);
}

// Pass C's MID form: one line per block (block-uniform line) and P = 2^k, so that register c
// of thread t holds column t + T c; when the line's plane box lies inside the middle half of
// the grid, P/4 .. 3P/4, only the registers c = 4 .. 11 hold box columns, and the inverse row
// transform's other outputs are unused.  (The same form of pass A, whose forward transform
// would take known zeros, measured slower: 9.85 -> 10.13 ms against 9.66 -> 9.45 ms here.)
template <int P, bool SHIFT>
__host__ __device__ constexpr bool mid_form_ok() {
  return !SHIFT && !Fft<P>::R3 && RowCfg<P>::G == 1;
}

// The box of line `li`'s plane inside the grid's middle half P/4 .. 3P/4 (false for lines past
// the end and, in HOLO_BOUNDS_CHECK builds, for bad line-table entries).
template <int P>
__device__ __forceinline__ bool line_box_mid(const PassArgs& a, int li) {
  if (li >= a.nlines) return false;
  const int2 L = __ldg(a.lines + a.line0 + li);
  if (kBoundsCheck && !line_ok(a, L.x, L.y, P)) return false;
  const PlaneDesc d = a.planes[L.x];
  return d.bx0 >= P / 4 && d.bx0 + d.bxs <= 3 * P / 4;
}

// Chirp exp(-i pi lambda z f^2)/P is even in the signed frequency, so a table of the
// P/2 + 1 non-negative frequencies suffices: entry f for f <= P/2, entry P - f above.
template <int P>
__device__ __forceinline__ float2 chirp_half(const float2* __restrict__ tab, int f) {
  const int i = f <= P / 2 ? f : P - f;
  return tab[Fft<P>::HW ? spad(i) : i];
}

// chirp_half at the frequencies fpos(t, c) held by thread t after the forward transform.
// For P = 2^k these are b + T c (b the thread's base, below T): entry b + T c for c < 8 and
// entry (T - b) + T (15 - c) for c >= 8 (the P/2 entry included), and at P = 4096 the padded
// index spad of either is linear in c with step T + T/16 (T = 256).  So two per-thread offsets
// make every lookup one shared-memory load at a constant offset.  P = 3 * 2^k keeps
// chirp_half.
template <int P, bool R3 = Fft<P>::R3>
struct ChirpAt {
  const float2* tab;
  int t;
  __device__ __forceinline__ ChirpAt(const float2* tb, int tt) : tab(tb), t(tt) {}
  __device__ __forceinline__ float2 operator()(int c) const {
    return chirp_half<P>(tab, Fft<P>::fpos(t, c));
  }
};
template <int P>
struct ChirpAt<P, false> {
  using F = Fft<P>;
  static constexpr int K = F::HW ? F::T + F::T / 16 : F::T;
  const float2* tab;
  int lo, hi;
  __device__ __forceinline__ ChirpAt(const float2* tb, int t) : tab(tb) {
    const int b = F::fpos(t, 0);
    lo = F::HW ? spad(b) : b;
    hi = F::HW ? spad(F::T - b) : F::T - b;
  }
  __device__ __forceinline__ float2 operator()(int c) const {
    return c < 8 ? tab[lo + K * c] : tab[hi + K * (15 - c)];
  }
};

// Copy the half chirp table of distance j into shared memory (block-wide).
template <int P>
__device__ __forceinline__ void load_chirp_half(float2* dst, const float2* __restrict__ src) {
  for (int i = threadIdx.x; i <= P / 2; i += blockDim.x) dst[Fft<P>::HW ? spad(i) : i] = src[i];
}

// ------------------------------------------------------------------ generic D-step

// One "FFT -> chirp -> inverse FFT" per line, lines = rows (COLS = false) or columns.
template <int P, bool COLS>
__global__ void __launch_bounds__(COLS ? ColCfg<P>::NT : RowCfg<P>::NT)
k_line_dstep(LineArgs a, const float2* __restrict__ gtw) {
  using F = Fft<P>;
  using H = SmemHead<P>;
  constexpr int G = COLS ? ColCfg<P>::C : RowCfg<P>::G;
  constexpr int LS = COLS ? ColCfg<P>::LS : RowCfg<P>::LS;
  extern __shared__ float2 smem[];
  float2* roots = smem;
  float2* chs = smem + H::ROOTS;
  const int g = COLS ? (int)(threadIdx.x % G) : (int)(threadIdx.x / F::T);
  const int t = COLS ? (int)(threadIdx.x / G) : (int)(threadIdx.x % F::T);
  float2* sm = smem + H::WORDS + g * LS;
  load_roots<P>(roots, gtw);
  load_chirp_half<P>(chs, a.chirp);
  const TwRoots tw{roots};
  const ChirpAt<P> cat(chs, t);
  for (int base = blockIdx.x * G; base < a.nlines; base += gridDim.x * G) {
    const int line = base + g;
    const bool valid = line < a.nlines;
    const float2* in = a.in + (long long)line * a.in_line_stride;
    float2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rel = F::pos(t, c) - a.in_lo;
      v[c] = (valid && (unsigned)rel < (unsigned)a.in_len) ? in[(long long)rel * a.in_step]
                                                           : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float2 ch = cat(c);
      v[c] = a.conj_chirp ? cmulc(v[c], ch) : cmul(v[c], ch);
    }
    fft_inv_with<P>(v, sm, tw, t, SyncBlock());
    float2* out = a.out + (long long)line * a.out_line_stride;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rel = F::pos(t, c) - a.out_lo;
      if (valid && (unsigned)rel < (unsigned)a.out_len) {
        float2* o = out + (long long)rel * a.out_step;
        float2 r = cscale(v[c], a.alpha);
        if (a.accumulate) r = cadd(r, *o);
        *o = r;
      }
    }
  }
}

// The column stage of sum_s D_s(x_s): the rows of every source were propagated already (row
// FFT, chirp, inverse), so D_s = IFFT_y chirp_s FFT_y on columns and the sum needs one inverse
// per column: acc = sum_s chirp_s FFT_y(col_s), out (+)= alpha IFFT_y(acc).  Blocks own C
// columns at a time, as k_line_dstep's column form; the half chirp tables of all sources stay
// in shared memory after the twiddle roots.
template <int P>
__global__ void __launch_bounds__(ColCfg<P>::NT)
k_cols_sum(const __grid_constant__ SumArgs a, const float2* __restrict__ gtw) {
  using F = Fft<P>;
  using H = SmemHead<P>;
  constexpr int G = ColCfg<P>::C, LS = ColCfg<P>::LS;
  extern __shared__ float2 smem[];
  const int g = threadIdx.x % G, t = threadIdx.x / G;
  float2* chs = smem + H::ROOTS;
  float2* sm = smem + H::ROOTS + a.S * H::CHIRP + g * LS;
  load_roots<P>(smem, gtw);
  for (int s = 0; s < a.S; ++s) load_chirp_half<P>(chs + s * H::CHIRP, a.chirp[s]);
  const TwRoots tw{smem};
  for (int base = blockIdx.x * G; base < P; base += gridDim.x * G) {
    const int col = base + g;
    const bool valid = col < P;
    float2 acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = make_float2(0.f, 0.f);
    for (int s = 0; s < a.S; ++s) {
      const float2* in = a.in[s] + col;
      const int r_lo = a.r_lo[s], rows = a.rows[s];
      float2 v[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int rel = F::pos(t, c) - r_lo;
        v[c] = (valid && (unsigned)rel < (unsigned)rows) ? in[(long long)rel * P]
                                                         : make_float2(0.f, 0.f);
      }
      // the exchange buffer is free once every thread finished the previous transform
      __syncthreads();
      fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
      const ChirpAt<P> cat(chs + s * H::CHIRP, t);
#pragma unroll
      for (int c = 0; c < 16; ++c)
        acc[c] = cadd(acc[c], a.conj_chirp ? cmulc(v[c], cat(c)) : cmul(v[c], cat(c)));
    }
    __syncthreads();
    fft_inv_with<P>(acc, sm, tw, t, SyncBlock());
    if (valid) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        float2* o = a.out + (long long)F::pos(t, c) * P + col;
        float2 r = cscale(acc[c], a.alpha);
        if (a.accumulate) r = cadd(r, *o);
        *o = r;
      }
    }
    __syncthreads();
  }
}

// Load the half chirp of distance j unless it is already resident (block-uniform j).
template <int P>
__device__ __forceinline__ void ensure_chirp(float2* chs, const float2* __restrict__ tables, int j,
                                             int& jcur) {
  if (j != jcur) {
    __syncthreads();
    load_chirp_half<P>(chs, tables + (long long)j * P);
    jcur = j;
  }
}

// ------------------------------------------------------------------ pass A

// Chirp table of distance j of problem `key` resident in shared memory: loaded unless the
// block's resident table already is that one (block-uniform arguments).
template <int P>
__device__ __forceinline__ void ensure_chirp_key(float2* chs, const float2* __restrict__ tables,
                                                 int j, int key, int& cur) {
  if (key != cur) {
    __syncthreads();
    load_chirp_half<P>(chs, tables + (long long)j * P);
    cur = key;
  }
}

// One block-step of pass A: the lines [base, base + G) of the problem `a` (indices relative
// to a.line0; lines past a.nlines are idle), one line per thread group.  `next` is the base of
// the block's next step in the same problem (its lines are prefetched into L2), or -1.  The
// resident chirp table is identified by pkey * 16 + distance (pkey: the problem's index in a
// batch, 0 for a single problem).
template <int P, bool SHIFT, bool HALF = false, class Args>
__device__ __forceinline__ void pass_a_step(const Args& a, int base, int next, float2* smem,
                                            const TwRoots& tw, int pkey, int& jcur) {
  using F = Fft<P>;
  using R = RowCfg<P>;
  using H = SmemHead<P>;
  float2* chs = smem + H::ROOTS;
  const int g = threadIdx.x / F::T, t = threadIdx.x % F::T;
  float2* sm = smem + H::WORDS + g * R::LS;
  const int n = a.n, lo = P / 2 - n / 2;
  float2* rmix = smem + H::WORDS + R::G * R::LS + g * n;  // [n] per line group
  const int p_lo = a.k0 * a.J;
  {
    const int li = base + g;
    bool valid = li < a.nlines;
    const int line = a.line0 + (valid ? li : 0);
    const int2 L = __ldg(a.lines + line);
    int gp = L.x, i = L.y;
    if constexpr (kBoundsCheck) {
      if (!line_ok(a, gp, i, P)) {
        if (valid) flag_bounds(a.err);
        valid = false;
        gp = p_lo;
        i = 0;
      }
    }
    const int lp = gp - p_lo, kl = lp / a.J, j = lp % a.J;
    const PlaneDesc d = a.planes[gp];
    const Tap yt = a.ytap[(long long)gp * a.tap_stride + i];
    const Tap* xt = a.xtap + (long long)gp * a.tap_stride;
    const float2* psi = a.psi + (long long)kl * n * n;
    const float2* prow = a.pj + ((long long)j * P + d.by0 + i) * P;
    float2* wrow = a.gkbuf + (long long)lp * a.gkstride + (long long)i * d.bxs;
    // lines of one block may belong to different distances only when G > 1; the chirp
    // table then follows the distance of the block's first line (block-uniform) and the
    // other lines read the chirp from global memory.
    int jb = (__ldg(a.lines + a.line0 + base).x - p_lo) % a.J;
    if (kBoundsCheck && (jb < 0 || jb >= a.J)) jb = 0;
    // the line's two object rows mixed with its row tap, into shared memory:
    //   r[ix] = (1 - fy) (psi[iy0][ix] - ext) + fy (psi[iy0 + 1][ix] - ext)
    // (rows outside psi dropped); the x-interpolation below reads r, so each object pixel
    // costs two coalesced, independent loads instead of four dependent gathers per position
    if (valid) {
      const bool r0 = (unsigned)yt.i0 < (unsigned)n, r1 = (unsigned)(yt.i0 + 1) < (unsigned)n;
      const float wy0 = 1.f - yt.f, wy1 = yt.f;
      const float2* p0 = psi + (long long)(r0 ? yt.i0 : 0) * n;
      const float2* p1 = psi + (long long)(r1 ? yt.i0 + 1 : 0) * n;
      for (int ix = t; ix < n; ix += F::T) {
        float2 r = make_float2(0.f, 0.f);
        if (r0) {
          const float2 q = __ldg(p0 + ix);
          r.x = wy0 * (q.x - a.ext);
          r.y = wy0 * q.y;
        }
        if (r1) {
          const float2 q = __ldg(p1 + ix);
          r.x = fmaf(wy1, q.x - a.ext, r.x);
          r.y = fmaf(wy1, q.y, r.y);
        }
        rmix[ix] = r;
      }
    }
    __syncthreads();
    float2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int X = F::pos(t, c), rel = X - d.bx0;
      float2 x = make_float2(0.f, 0.f);
      if (valid && (unsigned)rel < (unsigned)d.bxs) {
        const Tap xtp = xt[rel];
        float2 w = make_float2(0.f, 0.f);
        if ((unsigned)xtp.i0 < (unsigned)n) {
          const float2 r = rmix[xtp.i0];
          w.x = (1.f - xtp.f) * r.x;
          w.y = (1.f - xtp.f) * r.y;
        }
        if ((unsigned)(xtp.i0 + 1) < (unsigned)n) {
          const float2 r = rmix[xtp.i0 + 1];
          w.x = fmaf(xtp.f, r.x, w.x);
          w.y = fmaf(xtp.f, r.y, w.y);
        }
        if (SHIFT) w.x += a.ext;  // full-grid form: w = R' psi
        wrow[rel] = w;
        x = cmul(__ldg(prow + X), w);
      }
      v[c] = x;
    }
    // the next line of this thread group: its probe row and its two object rows go to L2 now
    // (one bulk request each, issued by the line's first thread)
    if (t == 0 && next >= 0 && next + g < a.nlines) {
      const int2 NL = __ldg(a.lines + a.line0 + next + g);
      // (a bad entry is flagged when its own line runs)
      if (!kBoundsCheck || line_ok(a, NL.x, NL.y, P)) {
      const int nlp = NL.x - p_lo;
      const PlaneDesc nd = a.planes[NL.x];
      const Tap nyt = a.ytap[(long long)NL.x * a.tap_stride + NL.y];
      l2_prefetch_bulk(a.pj + ((long long)(nlp % a.J) * P + nd.by0 + NL.y) * P + nd.bx0,
                       nd.bxs * (uint32_t)sizeof(float2));
      const float2* npsi = a.psi + (long long)(nlp / a.J) * n * n;
      if ((unsigned)nyt.i0 < (unsigned)n)
        l2_prefetch_bulk(npsi + (long long)nyt.i0 * n, n * (uint32_t)sizeof(float2));
      if ((unsigned)(nyt.i0 + 1) < (unsigned)n)
        l2_prefetch_bulk(npsi + (long long)(nyt.i0 + 1) * n, n * (uint32_t)sizeof(float2));
      }
    }
    ensure_chirp_key<P>(chs, a.chirp_zhat, R::G == 1 ? j : jb, pkey * 16 + (R::G == 1 ? j : jb),
                        jcur);
    __syncthreads();
    fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
    const bool own = R::G == 1 || pkey * 16 + j == jcur;
    const float2* chg = a.chirp_zhat + (long long)j * P;
    const ChirpAt<P> cat(chs, t);
    const float2* rmp = SHIFT ? a.ramp_x + (long long)gp * P : nullptr;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int f = F::fpos(t, c);
      v[c] = cmul(v[c], own ? cat(c) : __ldg(chg + f));
      if (SHIFT) v[c] = cmul(v[c], __ldg(rmp + f));
    }
    fft_inv_with<P>(v, sm, tw, t, SyncBlock());
    float2* yrow = a.ybuf + (long long)lp * a.ystride + (long long)i * n;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rel = F::pos(t, c) - lo;
      // HALF (n = P/2, P = 2^k >= 1024): the crop columns are those of registers 4 .. 11
      if (valid && (HALF ? (c >= 4 && c < 12) : (unsigned)rel < (unsigned)n)) yrow[rel] = v[c];
    }
  }
}

template <int P, bool SHIFT, bool HALF = false>
__global__ void __launch_bounds__(RowCfg<P>::NT, RowCfg<P>::MINB)
k_pass_a(const __grid_constant__ PassArgs a) {
  extern __shared__ float2 smem[];
  load_roots<P>(smem, a.twiddles);
  const TwRoots tw{smem};
  int jcur = -1;
  const int step = gridDim.x * RowCfg<P>::G;
  for (int base = blockIdx.x * RowCfg<P>::G; base < a.nlines; base += step)
    pass_a_step<P, SHIFT, HALF>(a, base, base + step < a.nlines ? base + step : -1, smem, tw, 0,
                                jcur);
}

// Pass A of several problems of line length P in one persistent launch: items {problem,
// base} of G lines each, walked by the blocks in a grid-stride loop (args: one PassArgs per
// problem, in device memory).
template <int P, bool SHIFT>
__global__ void __launch_bounds__(RowCfg<P>::NT, RowCfg<P>::MINB)
k_pass_a_multi(const PassArgs* __restrict__ args, const int2* __restrict__ items, int nitems) {
  extern __shared__ float2 smem[];
  load_roots<P>(smem, args[items[0].x].twiddles);  // every item has this P
  const TwRoots tw{smem};
  int jcur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    int next = -1;
    if (it + (int)gridDim.x < nitems) {
      const int2 ni = items[it + gridDim.x];
      if (ni.x == item.x) next = ni.y;
    }
    pass_a_step<P, SHIFT>(args[item.x], item.y, next, smem, tw, item.x, jcur);
  }
}

// ------------------------------------------------------------------ pass B

// Y stage of pass B: whole TMA boxes covering `rows` box rows of C columns.
template <int P>
size_t pass_b_stage_bytes(int rows) {
  return (size_t)((rows + kStageBox - 1) / kStageBox) * kStageBox * ColCfg<P>::C * sizeof(float2);
}

// Shared memory of pass B: head, C exchange lines, the reference field slice b[n][C] and
// the residual sum S[n][C] of the block's column group; with srows > 0 also the Y stage
// for planes of up to srows box rows (128-byte aligned).
template <int P>
size_t pass_b_smem(int n, int srows = 0) {
  const size_t base =
      (size_t)(SmemHead<P>::WORDS + ColCfg<P>::C * ColCfg<P>::LS + 2 * n * ColCfg<P>::C) *
      sizeof(float2);
  return srows > 0 ? base + 128 + pass_b_stage_bytes<P>(srows) : base;
}

// Pass B's Y stage: thread 0 arms the barrier and loads the tile of plane (kl, j) for
// column group cg (every box of the plane's box rows; rows past them are not read).
template <int P>
__device__ __forceinline__ void stage_y(const PassArgs& a, float2* stg, uint64_t* bar, int cg,
                                        int j, int kl) {
  constexpr int C = ColCfg<P>::C;
  const int bys = a.planes[(long long)(a.k0 + kl) * a.J + j].bys;
  const int nb = (bys + kStageBox - 1) / kStageBox;
  const int row0 = (kl * a.J + j) * a.yrows;
  mbar_expect_tx(bar, (uint32_t)(nb * kStageBox * C * sizeof(float2)));
  for (int b = 0; b < nb; ++b)
    tma_load_2d(stg + b * kStageBox * C, a.ymap, 2 * C * cg, row0 + b * kStageBox, bar);
}

// Each block owns whole column groups (C adjacent detector columns) and walks every plane
// of the chunk for them, distance-major: the columns of b = C D_{zeta_0} q are read once,
// and S = sum_kj r_kj is accumulated in shared memory in a fixed order and written once
// (with the reference residual) as the source of the ext-part of grad_q.  Every S / b slot
// is owned by one thread (its crop rows of its column), so no barrier guards them.
// The work of block `bid` of a pass-B grid of `nblk` blocks for the problem `a`: column groups
// bid, bid + nblk, ...; its FP64 loss partial goes to a.loss_part[bid].  The caller has loaded
// the twiddle roots at the head of shared memory and, for a staged problem, initialised the
// Y-stage barrier.  The resident chirp table is identified by pkey * 16 + distance.  Returns
// false when a bounded Y-stage wait gave up (the problem's error word is then set).  TSPLIT
// compiles in the split of a partial last round (a.pb_split == 2); without it the block's
// work is whole groups only and the segment bookkeeping folds away.
template <int P, bool ADJ, bool SHIFT, bool TSPLIT = false, bool HALF = false>
__device__ __forceinline__ bool pass_b_run(const PassArgs& a, int bid, int nblk, float2* smem,
                                           const TwRoots& tw, double* red, uint64_t* ybarp,
                                           uint32_t& yphase, int pkey, int& jcur) {
  using F = Fft<P>;
  using Cc = ColCfg<P>;
  using H = SmemHead<P>;
  constexpr int C = Cc::C;
  float2* chs = smem + H::ROOTS;
  const int g = threadIdx.x % C, t = threadIdx.x / C;
  const ChirpAt<P> cat(chs, t);
  float2* sm = smem + H::WORDS + g * Cc::LS;
  const int n = a.n, lo = P / 2 - n / 2;
  // HALF: n = P/2 with P = 2^k >= 1024, so the crop rows P/4 .. 3P/4 held by register c are
  // those of c = 4 .. 11 exactly and C divides n (every column of a group is in the crop); the
  // compiler then drops the checks, the zero inputs of the adjoint transform and the unused
  // outputs of the forward one
  static_assert(!HALF || (!F::R3 && P >= 1024), "the HALF form needs P = 2^k >= 1024");
  auto in_crop = [&](int c, int rr) {
    return HALF ? (c >= 4 && c < 12) : (unsigned)rr < (unsigned)n;
  };
  float2* sb = smem + H::WORDS + C * Cc::LS;
  float2* sS = sb + n * C;
  const int ngroups = (n + C - 1) / C;
  double dsum = 0.0;
  // Y stage: the tile of the block's next plane is in flight while the current one computes
  const bool staged = a.ymap != nullptr;
  float2* stg = reinterpret_cast<float2*>((reinterpret_cast<uintptr_t>(sS + n * C) + 127) &
                                          ~static_cast<uintptr_t>(127));
  // The block's work as segments {column group cg, planes [p0, p1)} with the planes in
  // (distance, angle) order p = j * nk + kl: whole groups bid, bid + nblk, ...; with the last
  // round split (a.pb_split == 2), the full rounds' whole groups and then the block's even share
  // of the last round's (group, plane) items, whose residual sums go to the block's slots.
  const int per = a.J * a.nk;
  const bool tsplit = TSPLIT && a.pb_split == 2 && ngroups % nblk != 0;
  const int rounds = tsplit ? ngroups / nblk : (ngroups - bid + nblk - 1) / nblk;
  const long long titems = tsplit ? (long long)(ngroups - rounds * nblk) * per : 0;
  const long long ti0 = titems * bid / nblk, ti1 = titems * (bid + 1) / nblk;
  auto segment = [&](int sg, int& gcg, int& q0, int& q1) -> bool {
    if (sg < rounds) {
      gcg = bid + sg * nblk;
      q0 = 0;
      q1 = per;
      return true;
    }
    if (!TSPLIT) return false;
    const long long tg = ti0 / per + (sg - rounds), g0 = tg * per;
    if (ti0 >= ti1 || g0 >= ti1) return false;
    gcg = rounds * nblk + (int)tg;
    q0 = (int)(ti0 > g0 ? ti0 - g0 : 0);
    q1 = (int)(ti1 - g0 < per ? ti1 - g0 : per);
    return true;
  };
  {
    int c0, q0, q1;
    if (staged && threadIdx.x == 0 && segment(0, c0, q0, q1))
      stage_y<P>(a, stg, ybarp, c0, q0 / a.nk, q0 % a.nk);
  }
  int cg, p0, p1;
  for (int sg = 0; segment(sg, cg, p0, p1); ++sg) {
    const int col = cg * C + g;
    const bool valid = HALF || col < n;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rr = F::pos(t, c) - lo;
      if (in_crop(c, rr)) {
        sb[rr * C + g] = (valid && a.ext != 0.f) ? __ldg(a.bref + (long long)rr * n + col)
                                                 : make_float2(0.f, 0.f);
        if (ADJ) sS[rr * C + g] = make_float2(0.f, 0.f);
      }
    }
    for (int pp = p0; pp < p1; ++pp) {
      const int j = pp / a.nk, kl = pp - j * a.nk;
      ensure_chirp_key<P>(chs, a.chirp_zhat, j, pkey * 16 + j, jcur);
      {
        const int lp = kl * a.J + j;
        const long long gplane = (long long)(a.k0 + kl) * a.J + j;
        PlaneDesc d = a.planes[gplane];
        if constexpr (kBoundsCheck) {
          if (!plane_box_ok(a, d, P)) {
            if (threadIdx.x == 0) flag_bounds(a.err);
            d.bys = 0;  // the plane's box rows are skipped
          }
        }
        // MID (n = P/2 form only): the plane's box rows lie in P/4 .. 3P/4, i.e. in the
        // registers c = 4 .. 11, so the forward column transform's other inputs are zero and the
        // adjoint transform's other outputs unused (planes run distance-major, so each form runs
        // in long stretches)
        auto plane = [&](auto mid) -> bool {
          constexpr bool MID = decltype(mid)::value;
          float2* yb = a.ybuf + (long long)lp * a.ystride;
          float2 v[16];
          if (staged) {
            const bool ok = mbar_wait(ybarp, yphase);
            yphase ^= 1;
  #pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int rel = F::pos(t, c) - d.by0;
              v[c] = ((!MID || (c >= 4 && c < 12)) && valid && (unsigned)rel < (unsigned)d.bys)
                         ? stg[rel * C + g]
                         : make_float2(0.f, 0.f);
            }
            // every thread has its tile entries: the stage is free for the next plane
            if (__syncthreads_or(!ok)) {
              if (threadIdx.x == 0) atomicOr(a.err, 1ull);
              return false;  // (leaves the plane; the caller returns)
            }
            if (threadIdx.x == 0) {
              int ncg = cg, np = pp + 1, n0, n1;
              bool more = np < p1;
              if (!more && segment(sg + 1, ncg, n0, n1)) {
                np = n0;
                more = true;
              }
              if (more) stage_y<P>(a, stg, ybarp, ncg, np / a.nk, np % a.nk);
            }
          } else {
  #pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int rel = F::pos(t, c) - d.by0;
              v[c] = ((!MID || (c >= 4 && c < 12)) && valid && (unsigned)rel < (unsigned)d.bys)
                         ? yb[(long long)rel * n + col]
                         : make_float2(0.f, 0.f);
            }
            __syncthreads();
          }
          fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
          // the data of the crop rows are fetched now, so the inverse transform hides their latency
          const float* ad =
              a.dblk + ((gplane - (long long)a.data_k0 * a.J) * a.dgroups + cg) * (long long)n * C;
          float dats[16];
  #pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int rr = F::pos(t, c) - lo;
            dats[c] = (valid && in_crop(c, rr)) ? __ldg(ad + rr * C + g) : 0.f;
          }
          const float2* rmp = SHIFT ? a.ramp_y + gplane * P : nullptr;
  #pragma unroll
          for (int c = 0; c < 16; ++c) {
            v[c] = cmul(v[c], cat(c));
            if (SHIFT) v[c] = cmul(v[c], __ldg(rmp + F::fpos(t, c)));
          }
          fft_inv_with<P>(v, sm, tw, t, SyncBlock());
          float2* uo = a.u_out ? a.u_out + (long long)lp * n * n : nullptr;
          float lsum = 0.f;
  #pragma unroll
          for (int c = 0; c < 16; ++c) {
            const int rr = F::pos(t, c) - lo;
            float2 r = make_float2(0.f, 0.f);
            if (valid && in_crop(c, rr)) {
              const long long e = (long long)rr * n + col;
              float2 u = v[c];
              const float2 b = sb[rr * C + g];
              u.x = fmaf(a.ext, b.x, u.x);
              u.y = fmaf(a.ext, b.y, u.y);
              const float dat = dats[c];
              const float i2 = fmaf(u.x, u.x, u.y * u.y);
              // F2: (|u| - a)^2, r = u - a u/|u| (u/|u| := 0 at |u| = 0);
              // F1: (|u|^2 - d)^2, r = 2 (|u|^2 - d) u
              float diff, s;
              if (a.functional) {
                diff = i2 - dat;
                s = 2.f * diff;
              } else {
                const float mag = sqrtf(i2);
                diff = mag - dat;
                s = mag > 0.f ? 1.f - __fdividef(dat, mag) : 0.f;
              }
              lsum = fmaf(diff, diff, lsum);
              if (uo) uo[e] = u;
              if (ADJ) {
                r = cscale(u, s);
                sS[rr * C + g] = cadd(sS[rr * C + g], r);
              }
            }
            v[c] = r;
          }
          dsum += (double)lsum;
          if constexpr (ADJ) {
            fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
  #pragma unroll
            for (int c = 0; c < 16; ++c) {
              v[c] = cmulc(v[c], cat(c));
              if (SHIFT) v[c] = cmulc(v[c], __ldg(rmp + F::fpos(t, c)));
            }
            fft_inv_with<P>(v, sm, tw, t, SyncBlock());
  #pragma unroll
            for (int c = 0; c < 16; ++c) {
              const int rel = F::pos(t, c) - d.by0;
              if ((!MID || (c >= 4 && c < 12)) && valid && (unsigned)rel < (unsigned)d.bys)
                yb[(long long)rel * n + col] = v[c];
            }
          }
          return true;
        };
        bool plane_ok;
        if constexpr (HALF) {
          if (d.by0 >= P / 4 && d.by0 + d.bys <= 3 * P / 4)
            plane_ok = plane(std::true_type{});
          else
            plane_ok = plane(std::false_type{});
        } else {
          plane_ok = plane(std::false_type{});
        }
        if (!plane_ok) return false;
      }
    }
    if constexpr (ADJ) {
      if (!TSPLIT || sg < rounds) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int rr = F::pos(t, c) - lo;
          if (valid && in_crop(c, rr)) {
            const long long e = (long long)rr * n + col;
            float2 acc = cscale(sS[rr * C + g], a.ext);
            if (a.tq_accumulate) acc = cadd(acc, a.tq[e]);
            if (a.rref) {
              const float2 q = __ldg(a.rref + e);
              acc.x = fmaf(a.wref, q.x, acc.x);
              acc.y = fmaf(a.wref, q.y, acc.y);
            }
            a.tq[e] = acc;
          }
        }
      } else if constexpr (TSPLIT) {
        // part of a last-round group: its partial residual sum goes to the block's slot
        // sg - rounds; k_pass_b_tail adds the slots of the group in block order into T
        float2* dst = a.tpart + ((long long)bid * a.tslots + (sg - rounds)) * n * C;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int rr = F::pos(t, c) - lo;
          if (in_crop(c, rr)) dst[rr * C + g] = sS[rr * C + g];
        }
      }
    }
  }
  const double s = block_sum_f64(dsum, red);
  if (threadIdx.x == 0) a.loss_part[bid] = s;
  return true;
}

template <int P, bool ADJ, bool SHIFT, bool TSPLIT = false, bool HALF = false>
__global__ void __launch_bounds__(ColCfg<P>::NT) k_pass_b(const __grid_constant__ PassArgs a) {
  extern __shared__ float2 smem[];
  __shared__ double red[32];
  __shared__ uint64_t ybar;
  load_roots<P>(smem, a.twiddles);
  const TwRoots tw{smem};
  if (a.ymap != nullptr) {
    if (threadIdx.x == 0) mbar_init(&ybar);
    __syncthreads();
  }
  uint32_t yphase = 0;
  int jcur = -1;
  pass_b_run<P, ADJ, SHIFT, TSPLIT, HALF>(a, blockIdx.x, gridDim.x, smem, tw, red, &ybar, yphase,
                                          0, jcur);
}

// Pass B of several problems of line length P in one persistent launch: items {problem, b},
// b < the problem's own pass-B grid (a.pb_blocks), each the work of block b of that grid, so
// every problem's results (loss partials included) are those of its own launch bit for bit.
// A Y-stage wait that gives up sets the error word of every problem of the launch.
template <int P, bool ADJ, bool SHIFT>
__global__ void __launch_bounds__(ColCfg<P>::NT)
k_pass_b_multi(const PassArgs* __restrict__ args, const int2* __restrict__ items, int nitems,
               int nprob) {
  extern __shared__ float2 smem[];
  __shared__ double red[32];
  __shared__ uint64_t ybar;
  load_roots<P>(smem, args[items[0].x].twiddles);  // every item has this P
  const TwRoots tw{smem};
  if (threadIdx.x == 0) mbar_init(&ybar);
  __syncthreads();
  uint32_t yphase = 0;
  int jcur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const PassArgs& a = args[item.x];
    if (!pass_b_run<P, ADJ, SHIFT>(a, item.y, a.pb_blocks, smem, tw, red, &ybar, yphase, item.x,
                                   jcur)) {
      if (threadIdx.x == 0)
        for (int p = 0; p < nprob; ++p) atomicOr(args[p].err, 1ull);
      return;
    }
  }
}

// Pass B when the column groups do not fill the GPU a few times over (fewer than three full
// rounds): whole groups in rounds as k_pass_b, then the (group, plane) items of the last,
// partial round split evenly over all blocks in (group, distance, angle) order.  Each block
// leaves S of every group it touched in its own slot; k_pass_b_tail adds the slots in block
// order (a fixed order) into T.  The item body is k_pass_b's.
template <int P, bool ADJ, bool SHIFT>
__global__ void __launch_bounds__(ColCfg<P>::NT) k_pass_b_split(PassArgs a) {
  using F = Fft<P>;
  using Cc = ColCfg<P>;
  using H = SmemHead<P>;
  constexpr int C = Cc::C;
  extern __shared__ float2 smem[];
  __shared__ double red[32];
  float2* roots = smem;
  float2* chs = smem + H::ROOTS;
  const int g = threadIdx.x % C, t = threadIdx.x / C;
  const ChirpAt<P> cat(chs, t);
  float2* sm = smem + H::WORDS + g * Cc::LS;
  const int n = a.n, lo = P / 2 - n / 2;
  float2* sb = smem + H::WORDS + C * Cc::LS;
  float2* sS = sb + n * C;
  load_roots<P>(roots, a.twiddles);
  const TwRoots tw{roots};
  const int ngroups = (n + C - 1) / C;
  double dsum = 0.0;
  int jcur = -1;

  auto begin_group = [&](int cg) {
    const int col = cg * C + g;
    const bool valid = col < n;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rr = F::pos(t, c) - lo;
      if ((unsigned)rr < (unsigned)n) {
        sb[rr * C + g] = (valid && a.ext != 0.f) ? __ldg(a.bref + (long long)rr * n + col)
                                                 : make_float2(0.f, 0.f);
        if (ADJ) sS[rr * C + g] = make_float2(0.f, 0.f);
      }
    }
  };
  auto item = [&](int cg, int j, int kl) {
    const int col = cg * C + g;
    const bool valid = col < n;
    const int lp = kl * a.J + j;
    const long long gplane = (long long)(a.k0 + kl) * a.J + j;
    PlaneDesc d = a.planes[gplane];
    if constexpr (kBoundsCheck) {
      if (!plane_box_ok(a, d, P)) {
        if (threadIdx.x == 0) flag_bounds(a.err);
        d.bys = 0;  // the plane's box rows are skipped
      }
    }
    float2* yb = a.ybuf + (long long)lp * a.ystride;
    float2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rel = F::pos(t, c) - d.by0;
      v[c] = (valid && (unsigned)rel < (unsigned)d.bys) ? yb[(long long)rel * n + col]
                                                         : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
    // the data of the crop rows are fetched now, so the inverse transform hides their latency
    const float* ad =
        a.dblk + ((gplane - (long long)a.data_k0 * a.J) * a.dgroups + cg) * (long long)n * C;
    float dats[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rr = F::pos(t, c) - lo;
      dats[c] = (valid && (unsigned)rr < (unsigned)n) ? __ldg(ad + rr * C + g) : 0.f;
    }
    const float2* rmp = SHIFT ? a.ramp_y + gplane * P : nullptr;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      v[c] = cmul(v[c], cat(c));
      if (SHIFT) v[c] = cmul(v[c], __ldg(rmp + F::fpos(t, c)));
    }
    fft_inv_with<P>(v, sm, tw, t, SyncBlock());
    float2* uo = a.u_out ? a.u_out + (long long)lp * n * n : nullptr;
    float lsum = 0.f;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rr = F::pos(t, c) - lo;
      float2 r = make_float2(0.f, 0.f);
      if (valid && (unsigned)rr < (unsigned)n) {
        const long long e = (long long)rr * n + col;
        float2 u = v[c];
        const float2 b = sb[rr * C + g];
        u.x = fmaf(a.ext, b.x, u.x);
        u.y = fmaf(a.ext, b.y, u.y);
        const float dat = dats[c];
        const float i2 = fmaf(u.x, u.x, u.y * u.y);
        float diff, s;
        if (a.functional) {
          diff = i2 - dat;
          s = 2.f * diff;
        } else {
          const float mag = sqrtf(i2);
          diff = mag - dat;
          s = mag > 0.f ? 1.f - __fdividef(dat, mag) : 0.f;
        }
        lsum = fmaf(diff, diff, lsum);
        if (uo) uo[e] = u;
        if (ADJ) {
          r = cscale(u, s);
          sS[rr * C + g] = cadd(sS[rr * C + g], r);
        }
      }
      v[c] = r;
    }
    dsum += (double)lsum;
    if constexpr (ADJ) {
      fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        v[c] = cmulc(v[c], cat(c));
        if (SHIFT) v[c] = cmulc(v[c], __ldg(rmp + F::fpos(t, c)));
      }
      fft_inv_with<P>(v, sm, tw, t, SyncBlock());
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int rel = F::pos(t, c) - d.by0;
        if (valid && (unsigned)rel < (unsigned)d.bys) yb[(long long)rel * n + col] = v[c];
      }
    }
  };

  const int rounds = ngroups / gridDim.x;
  for (int m = 0; m < rounds; ++m) {
    const int cg = blockIdx.x + m * gridDim.x;
    begin_group(cg);
    for (int j = 0; j < a.J; ++j) {
      ensure_chirp<P>(chs, a.chirp_zhat, j, jcur);
      for (int kl = 0; kl < a.nk; ++kl) item(cg, j, kl);
    }
    if constexpr (ADJ) {
      const int col = cg * C + g;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int rr = F::pos(t, c) - lo;
        if (col < n && (unsigned)rr < (unsigned)n) {
          const long long e = (long long)rr * n + col;
          float2 acc = cscale(sS[rr * C + g], a.ext);
          if (a.tq_accumulate) acc = cadd(acc, a.tq[e]);
          if (a.rref) {
            const float2 q = __ldg(a.rref + e);
            acc.x = fmaf(a.wref, q.x, acc.x);
            acc.y = fmaf(a.wref, q.y, acc.y);
          }
          a.tq[e] = acc;
        }
      }
    }
  }
  const int tail = ngroups - rounds * gridDim.x;
  const long long per = (long long)a.J * a.nk;
  const long long titems = (long long)tail * per;
  const long long i0 = titems * blockIdx.x / gridDim.x, i1 = titems * (blockIdx.x + 1) / gridDim.x;
  int slot = 0;
  for (long long it = i0; it < i1; ++slot) {
    const int tg = (int)(it / per);
    const long long pend = min(per, i1 - (long long)tg * per);
    const int cg = rounds * gridDim.x + tg;
    begin_group(cg);
    for (long long p = it - (long long)tg * per; p < pend; ++p) {
      const int j = (int)(p / a.nk), kl = (int)(p - (long long)j * a.nk);
      ensure_chirp<P>(chs, a.chirp_zhat, j, jcur);
      item(cg, j, kl);
    }
    if constexpr (ADJ) {
      float2* dst = a.tpart + ((long long)blockIdx.x * a.tslots + slot) * n * C;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int rr = F::pos(t, c) - lo;
        if ((unsigned)rr < (unsigned)n) dst[rr * C + g] = sS[rr * C + g];
      }
    }
    it = (long long)tg * per + pend;
  }
  const double s = block_sum_f64(dsum, red);
  if (threadIdx.x == 0) a.loss_part[blockIdx.x] = s;
}

// T of the last round's column groups of k_pass_b_split: the slots of every block whose item
// range met the group, added in block order, then T = ext S (+ T) (+ w_ref r_ref) as in
// k_pass_b.  One block per tail group.
template <int P>
__global__ void k_pass_b_tail(PassArgs a, int nblocks) {
  constexpr int C = ColCfg<P>::C;
  const int n = a.n;
  const int ngroups = (n + C - 1) / C;
  const int rounds = ngroups / nblocks, tail = ngroups - rounds * nblocks;
  const long long per = (long long)a.J * a.nk, titems = (long long)tail * per;
  const int tg = blockIdx.x;
  if (tg >= tail) return;
  const int cg = rounds * nblocks + tg;
  const long long g0 = (long long)tg * per, g1 = g0 + per;
  // blocks whose ranges [titems b / nblocks, titems (b + 1) / nblocks) meet [g0, g1)
  const int blo = max(0, (int)(g0 * nblocks / titems) - 1);
  const int bhi = min(nblocks - 1, (int)(g1 * nblocks / titems) + 1);
  for (int e = threadIdx.x; e < n * C; e += blockDim.x) {
    const int rr = e / C, g = e % C, col = cg * C + g;
    float2 S = make_float2(0.f, 0.f);
    for (int b = blo; b <= bhi; ++b) {
      const long long i0 = titems * b / nblocks, i1 = titems * (b + 1) / nblocks;
      if (i1 <= g0 || i0 >= g1 || i0 >= i1) continue;
      const int slot = tg - (int)(i0 / per);
      S = cadd(S, a.tpart[((long long)b * a.tslots + slot) * n * C + e]);
    }
    if (col < n) {
      const long long ie = (long long)rr * n + col;
      float2 acc = cscale(S, a.ext);
      if (a.tq_accumulate) acc = cadd(acc, a.tq[ie]);
      if (a.rref) {
        const float2 q = __ldg(a.rref + ie);
        acc.x = fmaf(a.wref, q.x, acc.x);
        acc.y = fmaf(a.wref, q.y, acc.y);
      }
      a.tq[ie] = acc;
    }
  }
}

// ------------------------------------------------------------------ pass C

// Pass C over items {problem, base} of several problems (args in device memory), one
// block-step of G lines per item (MULTI = true; the single-problem kernel has its own loop).
// The resident chirp table is identified by problem * 16 + distance.
template <int P, bool SHIFT>
__device__ __forceinline__ void pass_c_items(const PassArgs* __restrict__ args,
                                             const int2* __restrict__ items, int nitems) {
  using F = Fft<P>;
  using R = RowCfg<P>;
  using H = SmemHead<P>;
  extern __shared__ float2 smem[];
  load_roots<P>(smem, args[items[0].x].twiddles);  // every item has this P
  const TwRoots tw{smem};
  float2* chs = smem + H::ROOTS;
  const int g = threadIdx.x / F::T, t = threadIdx.x % F::T;
  float2* sm = smem + H::WORDS + g * R::LS;
  int jcur = -1;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const int pkey = item.x, base = item.y;
    int next = -1;
    if (it + (int)gridDim.x < nitems) {
      const int2 ni = items[it + gridDim.x];
      if (ni.x == item.x) next = ni.y;
    }
    const PassArgs& a = args[pkey];
    const int n = a.n, lo = P / 2 - n / 2;
    const int p_lo = a.k0 * a.J;
    const int li = base + g;
    bool valid = li < a.nlines;
    const int line = a.line0 + (valid ? li : 0);
    const int2 L = __ldg(a.lines + line);
    int gp = L.x, i = L.y;
    if constexpr (kBoundsCheck) {
      if (!line_ok(a, gp, i, P)) {
        if (valid) flag_bounds(a.err);
        valid = false;
        gp = p_lo;
        i = 0;
      }
    }
    const int lp = gp - p_lo, j = lp % a.J;
    int jb = (__ldg(a.lines + a.line0 + base).x - p_lo) % a.J;
    if (kBoundsCheck && (jb < 0 || jb >= a.J)) jb = 0;
    float2* yrow = a.ybuf + (long long)lp * a.ystride + (long long)i * n;
    float2 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int rel = F::pos(t, c) - lo;
      v[c] = (valid && (unsigned)rel < (unsigned)n) ? yrow[rel] : make_float2(0.f, 0.f);
    }
    // the next line of this thread group: its adjoint-field row, probe row and conj(w) v row go
    // to L2 now (one bulk request each, issued by the line's first thread)
    if (t == 0 && next >= 0 && next + g < a.nlines) {
      const int2 NL = __ldg(a.lines + a.line0 + next + g);
      // (a bad entry is flagged when its own line runs)
      if (!kBoundsCheck || line_ok(a, NL.x, NL.y, P)) {
      const int nlp = NL.x - p_lo;
      const PlaneDesc nd = a.planes[NL.x];
      l2_prefetch_bulk(a.ybuf + (long long)nlp * a.ystride + (long long)NL.y * n,
                       n * (uint32_t)sizeof(float2));
      l2_prefetch_bulk(a.pj + ((long long)(nlp % a.J) * P + nd.by0 + NL.y) * P + nd.bx0,
                       nd.bxs * (uint32_t)sizeof(float2));
      l2_prefetch_bulk(a.gkbuf + (long long)nlp * a.gkstride + (long long)NL.y * nd.bxs,
                       nd.bxs * (uint32_t)sizeof(float2));
      }
    }
    ensure_chirp_key<P>(chs, a.chirp_zhat, R::G == 1 ? j : jb, pkey * 16 + (R::G == 1 ? j : jb),
                        jcur);
    __syncthreads();
    fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
    const bool own = R::G == 1 || pkey * 16 + j == jcur;
    const float2* chg = a.chirp_zhat + (long long)j * P;
    const ChirpAt<P> cat(chs, t);
    const float2* rmp = SHIFT ? a.ramp_x + (long long)gp * P : nullptr;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int f = F::fpos(t, c);
      v[c] = cmulc(v[c], own ? cat(c) : __ldg(chg + f));
      if (SHIFT) v[c] = cmulc(v[c], __ldg(rmp + f));
    }
    fft_inv_with<P>(v, sm, tw, t, SyncBlock());
    // v holds the adjoint field on this P-grid row; the exchange buffer is free.
    // The box holds w = R0(psi - ext) (R' psi in the SHIFT form) written by pass A; replace
    // it by conj(w) v.
    const PlaneDesc d = a.planes[gp];
    const float2* prow = a.pj + ((long long)j * P + d.by0 + i) * P;
    float2* gk = a.gkbuf + (long long)lp * a.gkstride + (long long)i * d.bxs;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int X = F::pos(t, c), rel = X - d.bx0;
      if (valid && (unsigned)rel < (unsigned)d.bxs) {
        sm[rel] = cconjmul(__ldg(prow + X), v[c]);
        gk[rel] = cconjmul(gk[rel], v[c]);
      }
    }
    __syncthreads();
    // x-transpose of the bilinear resample: h[ip] = w0 z[X0] + w1 z[X0 + 1] with the
    // transposed taps of this plane (same FP64-built weights as the forward taps).
    const AdjTap* xa = a.xadj + (long long)gp * n;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const int ip = F::pos(t, c);
      if (!valid || ip >= n) continue;
      const AdjTap at = xa[ip];
      float2 h = make_float2(0.f, 0.f);
      const int r0 = at.X0 - d.bx0;
      if (at.w0 != 0.f) {
        const float2 z = sm[r0];
        h.x = at.w0 * z.x;
        h.y = at.w0 * z.y;
      }
      if (at.w1 != 0.f) {
        const float2 z = sm[r0 + 1];
        h.x = fmaf(at.w1, z.x, h.x);
        h.y = fmaf(at.w1, z.y, h.y);
      }
      yrow[ip] = h;
    }
    __syncthreads();
  }
}

// The single-problem pass C keeps its own grid-stride loop over the lines: built on the shared
// body below it measured slower (more spills).
template <int P, bool SHIFT, bool HALF = false>
__global__ void __launch_bounds__(RowCfg<P>::NT, RowCfg<P>::MINB) k_pass_c(PassArgs a) {
  using F = Fft<P>;
  using R = RowCfg<P>;
  using H = SmemHead<P>;
  extern __shared__ float2 smem[];
  float2* roots = smem;
  float2* chs = smem + H::ROOTS;
  const int g = threadIdx.x / F::T, t = threadIdx.x % F::T;
  float2* sm = smem + H::WORDS + g * R::LS;
  load_roots<P>(roots, a.twiddles);
  const TwRoots tw{roots};
  const int n = a.n, lo = P / 2 - n / 2;
  const int p_lo = a.k0 * a.J;
  int jcur = -1;
  for (int base = blockIdx.x * R::G; base < a.nlines; base += gridDim.x * R::G) {
    // MID (see mid_form_ok): the box columns are those of registers 4 .. 11, so the inverse
    // transform's other outputs are unused
    auto line = [&](auto mid) {
      constexpr bool MID = decltype(mid)::value;
      const int li = base + g;
      bool valid = li < a.nlines;
      const int line = a.line0 + (valid ? li : 0);
      const int2 L = __ldg(a.lines + line);
      int gp = L.x, i = L.y;
      if constexpr (kBoundsCheck) {
        if (!line_ok(a, gp, i, P)) {
          if (valid) flag_bounds(a.err);
          valid = false;
          gp = p_lo;
          i = 0;
        }
      }
      const int lp = gp - p_lo, j = lp % a.J;
      int jb = (__ldg(a.lines + a.line0 + base).x - p_lo) % a.J;
      if (kBoundsCheck && (jb < 0 || jb >= a.J)) jb = 0;
      float2* yrow = a.ybuf + (long long)lp * a.ystride + (long long)i * n;
      float2 v[16];
  #pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int rel = F::pos(t, c) - lo;
        // HALF (n = P/2, P = 2^k >= 1024): the crop columns are those of registers 4 .. 11
        const bool in = HALF ? (c >= 4 && c < 12) : (unsigned)rel < (unsigned)n;
        v[c] = (valid && in) ? yrow[rel] : make_float2(0.f, 0.f);
      }
      // the next line of this thread group: its adjoint-field row, probe row and conj(w) v row go
      // to L2 now (one bulk request each, issued by the line's first thread)
      if (t == 0 && li + (int)gridDim.x * R::G < a.nlines) {
        const int2 NL = __ldg(a.lines + a.line0 + li + gridDim.x * R::G);
        // (a bad entry is flagged when its own line runs)
        if (!kBoundsCheck || line_ok(a, NL.x, NL.y, P)) {
          const int nlp = NL.x - p_lo;
          const PlaneDesc nd = a.planes[NL.x];
          l2_prefetch_bulk(a.ybuf + (long long)nlp * a.ystride + (long long)NL.y * n,
                           n * (uint32_t)sizeof(float2));
          l2_prefetch_bulk(a.pj + ((long long)(nlp % a.J) * P + nd.by0 + NL.y) * P + nd.bx0,
                           nd.bxs * (uint32_t)sizeof(float2));
          l2_prefetch_bulk(a.gkbuf + (long long)nlp * a.gkstride + (long long)NL.y * nd.bxs,
                           nd.bxs * (uint32_t)sizeof(float2));
        }
      }
      ensure_chirp<P>(chs, a.chirp_zhat, R::G == 1 ? j : jb, jcur);
      __syncthreads();
      fft_fwd_with<P>(v, sm, tw, t, SyncBlock());
      const bool own = R::G == 1 || j == jcur;
      const float2* chg = a.chirp_zhat + (long long)j * P;
      const ChirpAt<P> cat(chs, t);
      const float2* rmp = SHIFT ? a.ramp_x + (long long)gp * P : nullptr;
  #pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int f = F::fpos(t, c);
        v[c] = cmulc(v[c], own ? cat(c) : __ldg(chg + f));
        if (SHIFT) v[c] = cmulc(v[c], __ldg(rmp + f));
      }
      fft_inv_with<P>(v, sm, tw, t, SyncBlock());
      // v holds the adjoint field on this P-grid row; the exchange buffer is free.
      // The box holds w = R0(psi - ext) (R' psi in the SHIFT form) written by pass A; replace
      // it by conj(w) v.
      const PlaneDesc d = a.planes[gp];
      const float2* prow = a.pj + ((long long)j * P + d.by0 + i) * P;
      float2* gk = a.gkbuf + (long long)lp * a.gkstride + (long long)i * d.bxs;
  #pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int X = F::pos(t, c), rel = X - d.bx0;
        if ((!MID || (c >= 4 && c < 12)) && valid && (unsigned)rel < (unsigned)d.bxs) {
          sm[rel] = cconjmul(__ldg(prow + X), v[c]);
          gk[rel] = cconjmul(gk[rel], v[c]);
        }
      }
      __syncthreads();
      // x-transpose of the bilinear resample: h[ip] = w0 z[X0] + w1 z[X0 + 1] with the
      // transposed taps of this plane (same FP64-built weights as the forward taps).
      const AdjTap* xa = a.xadj + (long long)gp * n;
  #pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int ip = F::pos(t, c);
        if (!valid || (HALF ? c >= 8 : ip >= n)) continue;
        const AdjTap at = xa[ip];
        float2 h = make_float2(0.f, 0.f);
        const int r0 = at.X0 - d.bx0;
        if (at.w0 != 0.f) {
          const float2 z = sm[r0];
          h.x = at.w0 * z.x;
          h.y = at.w0 * z.y;
        }
        if (at.w1 != 0.f) {
          const float2 z = sm[r0 + 1];
          h.x = fmaf(at.w1, z.x, h.x);
          h.y = fmaf(at.w1, z.y, h.y);
        }
        yrow[ip] = h;
      }
      __syncthreads();
    };
    if constexpr (mid_form_ok<P, SHIFT>()) {
      if (line_box_mid<P>(a, base))
        line(std::true_type{});
      else
        line(std::false_type{});
    } else {
      line(std::false_type{});
    }
  }
}

// Pass C of several problems of line length P in one persistent launch (items as
// k_pass_a_multi).
template <int P, bool SHIFT>
__global__ void __launch_bounds__(RowCfg<P>::NT, RowCfg<P>::MINB)
k_pass_c_multi(const PassArgs* __restrict__ args, const int2* __restrict__ items, int nitems) {
  pass_c_items<P, SHIFT>(args, items, nitems);
}

// ------------------------------------------------------------------ launchers

inline int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

// Persistent grid: as many blocks as can be resident at once, capped by the work.
template <class K>
int persistent_blocks(K kernel, int threads, size_t smem, long long items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  long long b = (long long)per_sm * sm_count();
  if (items < b) b = items;
  return (int)(b < 1 ? 1 : b);
}

// Persistent grid of a multi-problem launch: per_sm (or as many as fit) blocks per SM,
// capped by the items.
template <class K>
int multi_blocks(K kernel, int threads, size_t smem, int nitems, int per_sm) {
  int fit = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, kernel, threads, smem) != cudaSuccess ||
      fit < 1) {
    cudaGetLastError();
    fit = 1;
  }
  const int b = (per_sm > 0 && per_sm < fit ? per_sm : fit) * sm_count();
  return b < nitems ? b : (nitems > 0 ? nitems : 1);
}

template <int P, bool COLS>
cudaError_t launch_lines(const LineArgs& a, const float2* tw, cudaStream_t s) {
  constexpr int G = COLS ? ColCfg<P>::C : RowCfg<P>::G;
  constexpr int NT = COLS ? ColCfg<P>::NT : RowCfg<P>::NT;
  constexpr size_t SM = COLS ? ColCfg<P>::SMEM_BYTES : RowCfg<P>::SMEM_BYTES;
  if (a.nlines <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_line_dstep<P, COLS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM);
  if (e != cudaSuccess) return e;
  const int nb = persistent_blocks(k_line_dstep<P, COLS>, NT, SM, (a.nlines + G - 1) / G);
  k_line_dstep<P, COLS><<<nb, NT, SM, s>>>(a, tw);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_rows(const LineArgs& a, const float2* tw, cudaStream_t s) {
  return launch_lines<P, false>(a, tw, s);
}
template <int P>
cudaError_t launch_cols(const LineArgs& a, const float2* tw, cudaStream_t s) {
  return launch_lines<P, true>(a, tw, s);
}


// Pass A's shared memory: the row pass layout plus one mixed object row [n] per line.
template <int P>
size_t pass_a_smem(int n) {
  return RowCfg<P>::SMEM_BYTES + (size_t)RowCfg<P>::G * n * sizeof(float2);
}

template <int P, bool SHIFT, bool HALF = false>
cudaError_t launch_pass_a_form(const PassArgs& a, cudaStream_t s) {
  using R = RowCfg<P>;
  if (a.nlines <= 0) return cudaSuccess;
  const size_t sm = pass_a_smem<P>(a.n);
  cudaError_t e = cudaFuncSetAttribute(k_pass_a<P, SHIFT, HALF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int nb = multi_blocks(k_pass_a<P, SHIFT, HALF>, R::NT, sm, (a.nlines + R::G - 1) / R::G,
                              a.row_per_sm);
  k_pass_a<P, SHIFT, HALF><<<nb, R::NT, sm, s>>>(a);
  return cudaGetLastError();
}

// Lines with n = P/2 (P = 2^k >= 1024, no probe shifts) run the row passes' HALF forms, whose
// crop columns are fixed at compile time.
template <int P>
constexpr bool half_form_ok() {
  return !Fft<P>::R3 && P >= 1024;
}

template <int P>
cudaError_t launch_pass_a(const PassArgs& a, cudaStream_t s) {
  if (a.ramp_x) return launch_pass_a_form<P, true>(a, s);
  if constexpr (half_form_ok<P>())
    if (2 * a.n == P) return launch_pass_a_form<P, false, true>(a, s);
  return launch_pass_a_form<P, false>(a, s);
}

template <int P>
int pass_b_groups(int n) {
  return (n + ColCfg<P>::C - 1) / ColCfg<P>::C;
}

inline int max_dynamic_smem() {
  static int v = 0;
  if (!v) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (v <= 0) v = 48 * 1024;
  }
  return v;
}

template <int P>
size_t cols_sum_smem(int S) {
  return (size_t)(SmemHead<P>::ROOTS + S * SmemHead<P>::CHIRP + ColCfg<P>::C * ColCfg<P>::LS) *
         sizeof(float2);
}

template <int P>
int cols_sum_max() {
  const size_t cap = (size_t)max_dynamic_smem();
  int S = 0;
  while (S < kMaxSumSources && cols_sum_smem<P>(S + 1) <= cap) ++S;
  return S;
}

// cudaErrorNotSupported (nothing launched) when the sources' chirps do not fit.
template <int P>
cudaError_t launch_cols_sum(const SumArgs& a, const float2* tw, cudaStream_t s) {
  using Cc = ColCfg<P>;
  if (a.S < 1 || a.S > cols_sum_max<P>()) return cudaErrorNotSupported;
  const size_t sm = cols_sum_smem<P>(a.S);
  cudaError_t e = cudaFuncSetAttribute(k_cols_sum<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  const int nb = persistent_blocks(k_cols_sum<P>, Cc::NT, sm, (P + Cc::C - 1) / Cc::C);
  k_cols_sum<P><<<nb, Cc::NT, sm, s>>>(a, tw);
  return cudaGetLastError();
}

// rows: box rows of the Y stage (0: plain loads)
template <int P>
int pass_b_blocks(int items, int n, int rows) {
  using Cc = ColCfg<P>;
  const size_t sm = pass_b_smem<P>(n, rows);
  if (sm > (size_t)max_dynamic_smem()) return 0;
  cudaFuncSetAttribute(k_pass_b<P, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return persistent_blocks(k_pass_b<P, true, false>, Cc::NT, sm, items);
}

// The Y stage is used where the box is at most 2C x kStageBox floats wide (P >= 1024), the
// shared memory fits and pass B keeps its resident blocks per SM.
template <int P>
int pass_b_stage_ok(int n, int rows) {
  using Cc = ColCfg<P>;
  if (P < 1024 || rows <= 0 || 2 * Cc::C > kStageBox) return 0;
  const size_t s0 = pass_b_smem<P>(n), s1 = pass_b_smem<P>(n, rows);
  if (s1 > (size_t)max_dynamic_smem()) return 0;
  int b0 = 0, b1 = 0;
  if (cudaFuncSetAttribute(k_pass_b<P, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)s1) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, k_pass_b<P, true, false>, Cc::NT, s0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_pass_b<P, true, false>, Cc::NT, s1) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b1 >= 1 && b1 == b0 ? 1 : 0;
}

template <int P>
int pass_b_blocks_split(long long items, int n) {
  using Cc = ColCfg<P>;
  const size_t sm = pass_b_smem<P>(n);
  cudaFuncSetAttribute(k_pass_b_split<P, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sm);
  return persistent_blocks(k_pass_b_split<P, true, false>, Cc::NT, sm, items);
}

template <int P, bool ADJ, bool SHIFT>
cudaError_t launch_pass_b_split(const PassArgs& a, int nblocks, size_t sm, cudaStream_t s) {
  using Cc = ColCfg<P>;
  cudaError_t e = cudaFuncSetAttribute(k_pass_b_split<P, ADJ, SHIFT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_pass_b_split<P, ADJ, SHIFT><<<nblocks, Cc::NT, sm, s>>>(a);
  const int ngroups = (a.n + Cc::C - 1) / Cc::C, tail = ngroups - (ngroups / nblocks) * nblocks;
  if (ADJ && tail > 0) {
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pass_b_tail<P><<<tail, 256, 0, s>>>(a, nblocks);
  }
  return cudaGetLastError();
}

template <int P, bool ADJ, bool SHIFT, bool TSPLIT, bool HALF = false>
cudaError_t launch_pass_b_staged(const PassArgs& a, int nblocks, cudaStream_t s) {
  using Cc = ColCfg<P>;
  const size_t sm = pass_b_smem<P>(a.n, a.ymap ? a.max_box_rows : 0);
  cudaError_t e = cudaFuncSetAttribute(k_pass_b<P, ADJ, SHIFT, TSPLIT, HALF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_pass_b<P, ADJ, SHIFT, TSPLIT, HALF><<<nblocks, Cc::NT, sm, s>>>(a);
  const int ngroups = (a.n + Cc::C - 1) / Cc::C, tail = ngroups - (ngroups / nblocks) * nblocks;
  if (TSPLIT && tail > 0) {
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pass_b_tail<P><<<tail, 256, 0, s>>>(a, nblocks);
  }
  return cudaGetLastError();
}

// pb_split: 0 whole column groups per block; 1 the plane-split kernel (no Y stage); 2 the
// staged kernel with its last round split by planes, then the combine kernel.  The staged
// split is compiled for the gradient without probe shifts; the other forms run pb_split 2 as
// whole groups on the same grid.  Whole groups with n = P/2 (P = 2^k >= 1024, no probe
// shifts) run the HALF form, whose crop rows are fixed at compile time.
template <int P, bool ADJ, bool SHIFT>
cudaError_t launch_pass_b_form(const PassArgs& a, int nblocks, cudaStream_t s) {
  if (a.pb_split == 1) {
    PassArgs b = a;
    b.ymap = nullptr;
    return launch_pass_b_split<P, ADJ, SHIFT>(b, nblocks, pass_b_smem<P>(a.n), s);
  }
  if constexpr (ADJ && !SHIFT) {
    if (a.pb_split == 2) return launch_pass_b_staged<P, true, false, true>(a, nblocks, s);
  }
  if constexpr (!SHIFT && half_form_ok<P>()) {
    if (2 * a.n == P) return launch_pass_b_staged<P, ADJ, false, false, true>(a, nblocks, s);
  }
  return launch_pass_b_staged<P, ADJ, SHIFT, false>(a, nblocks, s);
}

// The SHIFT form (probe shifts) runs without the Y stage: its box is the whole grid.
template <int P>
cudaError_t launch_pass_b(const PassArgs& a, int adj, int nblocks, cudaStream_t s) {
  if (a.ramp_y) {
    PassArgs b = a;
    b.ymap = nullptr;
    return adj ? launch_pass_b_form<P, true, true>(b, nblocks, s)
               : launch_pass_b_form<P, false, true>(b, nblocks, s);
  }
  return adj ? launch_pass_b_form<P, true, false>(a, nblocks, s)
             : launch_pass_b_form<P, false, false>(a, nblocks, s);
}

template <int P, bool SHIFT, bool HALF = false>
cudaError_t launch_pass_c_form(const PassArgs& a, cudaStream_t s) {
  using R = RowCfg<P>;
  if (a.nlines <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_pass_c<P, SHIFT, HALF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)R::SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int nb = multi_blocks(k_pass_c<P, SHIFT, HALF>, R::NT, R::SMEM_BYTES,
                              (a.nlines + R::G - 1) / R::G, a.row_per_sm);
  k_pass_c<P, SHIFT, HALF><<<nb, R::NT, R::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_pass_c(const PassArgs& a, cudaStream_t s) {
  if (a.ramp_x) return launch_pass_c_form<P, true>(a, s);
  if constexpr (half_form_ok<P>())
    if (2 * a.n == P) return launch_pass_c_form<P, false, true>(a, s);
  return launch_pass_c_form<P, false>(a, s);
}

template <int P, bool SHIFT>
cudaError_t launch_rows_multi_form(int pass_c, const PassArgs* args, const int2* items,
                                   int nitems, int max_n, int per_sm, cudaStream_t s) {
  using R = RowCfg<P>;
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = pass_c ? R::SMEM_BYTES : pass_a_smem<P>(max_n);
  auto kern = pass_c ? k_pass_c_multi<P, SHIFT> : k_pass_a_multi<P, SHIFT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int nb = multi_blocks(kern, R::NT, sm, nitems, per_sm);
  kern<<<nb, R::NT, sm, s>>>(args, items, nitems);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_rows_multi(int pass_c, const PassArgs* args, const int2* items, int nitems,
                              int shift, int max_n, int per_sm, cudaStream_t s) {
  return shift ? launch_rows_multi_form<P, true>(pass_c, args, items, nitems, max_n, per_sm, s)
               : launch_rows_multi_form<P, false>(pass_c, args, items, nitems, max_n, per_sm, s);
}

template <int P, bool ADJ, bool SHIFT>
cudaError_t launch_pass_b_multi_form(const PassArgs* args, const int2* items, int nitems,
                                     int nprob, int max_n, int max_rows, int per_sm,
                                     cudaStream_t s) {
  using Cc = ColCfg<P>;
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = pass_b_smem<P>(max_n, max_rows);
  auto kern = k_pass_b_multi<P, ADJ, SHIFT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int nb = multi_blocks(kern, Cc::NT, sm, nitems, per_sm);
  kern<<<nb, Cc::NT, sm, s>>>(args, items, nitems, nprob);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_pass_b_multi(const PassArgs* args, const int2* items, int nitems, int nprob,
                                int adj, int shift, int max_n, int max_rows, int per_sm,
                                cudaStream_t s) {
  if (shift)
    return adj ? launch_pass_b_multi_form<P, true, true>(args, items, nitems, nprob, max_n, 0, per_sm, s)
               : launch_pass_b_multi_form<P, false, true>(args, items, nitems, nprob, max_n, 0, per_sm, s);
  return adj ? launch_pass_b_multi_form<P, true, false>(args, items, nitems, nprob, max_n, max_rows, per_sm, s)
             : launch_pass_b_multi_form<P, false, false>(args, items, nitems, nprob, max_n, max_rows, per_sm, s);
}

template <int P>
const Ops* make_ops() {
  static const Ops ops = {P,
                          launch_rows<P>,
                          launch_cols<P>,
                          launch_pass_a<P>,
                          launch_pass_b<P>,
                          launch_pass_c<P>,
                          pass_b_groups<P>,
                          pass_b_blocks<P>,
                          pass_b_blocks_split<P>,
                          pass_b_stage_ok<P>,
                          Fft<P>::TW,
                          ColCfg<P>::C,
                          RowCfg<P>::G,
                          launch_rows_multi<P>,
                          launch_pass_b_multi<P>,
                          launch_cols_sum<P>,
                          cols_sum_max<P>};
  return &ops;
}

}  // namespace holo

#define HOLO_INSTANTIATE(P) \
  namespace holo {          \
  const Ops* ops_##P() { return make_ops<P>(); } \
  }
