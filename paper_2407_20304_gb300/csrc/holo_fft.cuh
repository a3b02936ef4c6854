// Register + shared-memory FFT engine for one line of length P: a power of two >= 16, or
// three times one (P = 3 PB, PB >= 16).
//
// The Fresnel operator D_z (Appendix A, Eq. defPz/defGz) is a circular convolution on
// the P x P grid; with a separable chirp exp(-i pi lambda z (fx^2 + fy^2)) it factors into
// one pass over rows and one over columns, each "FFT -> chirp -> inverse FFT" along a
// line.  This header implements that line transform.
//
// Layout.  A line is held by T = P/16 threads, 16 complex values per thread: thread t,
// register c holds element t + T*c ("strided natural" layout).  The forward transform
// is a mixed-radix decimation in frequency with radices 16, 16, ..., 16, r (r in
// {2, 4, 8} when log2 P is not a multiple of 4); every stage is a DFT over one digit in
// registers followed by a twiddle and a shared-memory exchange.  The thread/register
// assignment of each stage is chosen so that the forward output is again in strided
// natural order (register rho of thread t holds frequency t + T*rho), so a pointwise
// multiplier in frequency needs no reordering and the inverse transform (the adjoint
// stages in reverse order) consumes that layout directly and returns the same layout.
//
// Exchanges write register k of thread t at t + T*k (contiguous per k) and read the
// next stage's digit; addresses are padded a -> a + a/16 so both phases avoid shared
// memory bank conflicts.  Twiddles come from a per-stage table in shared memory,
// indexed [k-1][mu] so that consecutive threads read consecutive entries.
//
// P = 3 PB.  The T = P/16 threads form three groups of TB = PB/16; thread t = q TB + i
// holds element i + TB c + PB q (pos).  The forward transform first takes one radix-3
// decimation-in-frequency step through shared memory: group q forms
//   y_q[n] = W_P^{n q} (x[n] + W_3^q x[n + PB] + W_3^{2q} x[n + 2 PB]),  n = i + TB c,
// which is one output of each of the PB three-point butterflies, then group q transforms
// y_q with the power-of-two engine above on its own third of the buffer.  Register rho of
// thread (q, i) then holds frequency 3 (i + TB rho) + q (fpos).  The inverse runs the
// adjoint steps in reverse order and returns the pos layout.
//
// Synchronisation: every thread of a line group calls the transform the same number of
// times; the Sync policy is a block-wide barrier or a named barrier per line group.  The
// buffer must be free when a transform starts.  It is free again when fft_inv returns; after
// fft_fwd at P = 4096 other thread groups may still read their rows of the last (group-local)
// exchange, so an fft_inv may follow directly (it starts on the same threads' rows) and any
// other use of the buffer needs a barrier first.

#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace holo {

// --------------------------------------------------------------------- complex helpers

// Packed two-lane FP32 add / subtract (PTX add/sub .f32x2, sm_100 and later): both
// components of a complex value in one instruction, with the same IEEE rounding as two scalar
// operations (outputs are bit-identical to the scalar form; the issue slots of the butterfly
// additions halve).  HOLO_SCALAR_COMPLEX selects the scalar form.
#if !defined(HOLO_SCALAR_COMPLEX)
__device__ __forceinline__ unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk(a)), "l"(pk(b)));
  return upk(d);
}
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// --------------------------------------------------------------------- shapes

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }
__host__ __device__ constexpr int ipow16(int s) { return s == 0 ? 1 : 16 * ipow16(s - 1); }

__device__ __forceinline__ int spad(int a) { return a + (a >> 4); }
__host__ __device__ constexpr int spad_c(int a) { return a + (a >> 4); }

__host__ __device__ constexpr bool is_pow2c(int x) { return x > 0 && (x & (x - 1)) == 0; }

template <int P_>
struct Fft {
  static constexpr int P = P_;
  static constexpr bool R3 = P % 3 == 0;           // one radix-3 step, then three sub-lines
  static constexpr int PB = R3 ? P / 3 : P;        // power-of-two (sub-)line length
  static_assert(is_pow2c(PB) && PB >= 16, "line length must be 2^k or 3 * 2^k with 2^k >= 16");
  static constexpr int LOG2 = ilog2c(PB);
  static constexpr int T = P / 16;                 // threads per line
  static constexpr int TB = PB / 16;               // threads per power-of-two sub-line
  static constexpr int N16 = LOG2 / 4;             // radix-16 stages
  static constexpr int RB = LOG2 % 4;              // bits of the final small stage (0: none)
  static constexpr int NST = N16 + (RB ? 1 : 0);   // number of stages
  static constexpr int RLAST = RB ? (1 << RB) : 16;
  static constexpr int SMEM = P + P / 16;          // padded exchange buffer, float2 entries
  // radix-16 stage s: prefix length L = 16^s, remaining length M = PB / 16^(s+1)
  __host__ __device__ static constexpr int L(int s) { return ipow16(s); }
  __host__ __device__ static constexpr int M(int s) { return PB / ipow16(s + 1); }
  __host__ __device__ static constexpr int tw_off(int s) {
    return s == 0 ? 0 : tw_off(s - 1) + (M(s - 1) > 1 ? 15 * M(s - 1) : 0);
  }
  static constexpr int TW_BASE = tw_off(N16);      // radix-16 twiddle entries (float2)
  // compact table of the roots W_PB^{mu L(s)} (k = 1 entries) of every twiddled stage
  __host__ __device__ static constexpr int roots_off(int s) {
    return s == 0 ? 0 : roots_off(s - 1) + (M(s - 1) > 1 ? M(s - 1) : 0);
  }
  static constexpr int ROOTS_BASE = roots_off(N16);
  // radix-3 step: W_P^n and W_P^{2n}, n < PB, appended to both tables
  static constexpr int TW = TW_BASE + (R3 ? 2 * PB : 0);
  static constexpr int ROOTS = ROOTS_BASE + (R3 ? 2 * PB : 0);
  // P = 4096: the exchange before the last radix-16 stage stays inside each group of 16
  // threads t = 16a .. 16a + 15 (which every kernel keeps in one warp), so it needs a warp
  // barrier only; the last stage then numbers its threads k1 + 16 a (see fwd_from).
  static constexpr bool HW = !R3 && RB == 0 && N16 == 3;
  static constexpr int HW_ROW = 17, HW_GROUP = 16 * 17;  // group region: 16 rows of 17
  // line element held in register c of thread t, and the frequency it holds after fft_fwd
  __host__ __device__ static constexpr int pos(int t, int c) {
    return R3 ? t % TB + TB * c + PB * (t / TB) : t + T * c;
  }
  __host__ __device__ static constexpr int fpos(int t, int c) {
    return R3 ? 3 * (t % TB + TB * c) + t / TB
              : (HW ? (t >> 4) + (T / 16) * (t & 15) + T * c : t + T * c);
  }
};

// --------------------------------------------------------------------- small DFTs

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 s = cadd(a, b), d = csub(a, b);
  a = s;
  b = d;
}

// natural order in, natural order out
template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
  const float2 s13 = cadd(x1, x3), e = csub(x1, x3);
  x0 = cadd(s02, s13);
  x2 = csub(s02, s13);
  // d02 +/- (-i e) forward, d02 +/- (i e) inverse, the swap folded into scalar adds
  const float2 p = make_float2(d02.x + e.y, d02.y - e.x), m = make_float2(d02.x - e.y, d02.y + e.x);
  x1 = INV ? m : p;
  x3 = INV ? p : m;
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  // radix-2 decimation in time over two DFT-4s
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  const float h = 0.70710678118654752f;
  // W8^1 = (1 - i)/sqrt2 forward, (1 + i)/sqrt2 inverse
  float2 t1 = INV ? make_float2((o1.x - o1.y) * h, (o1.x + o1.y) * h)
                  : make_float2((o1.x + o1.y) * h, (o1.y - o1.x) * h);
  float2 t2 = mul_mi<INV>(o2);
  // W8^3 = (-1 - i)/sqrt2 forward, (-1 + i)/sqrt2 inverse
  float2 t3 = INV ? make_float2((-o3.x - o3.y) * h, (o3.x - o3.y) * h)
                  : make_float2((o3.y - o3.x) * h, (-o3.x - o3.y) * h);
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

// W16^m as (cos, -sin) of 2 pi m / 16 (conjugated for the inverse)
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
  float2 w;
  switch (m) {
    case 1: w = make_float2(c1, -s1); break;
    case 2: w = make_float2(h, -h); break;
    case 3: w = make_float2(s1, -c1); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 6: w = make_float2(-h, -h); break;
    case 9: w = make_float2(-c1, s1); break;
    default: w = make_float2(1.f, 0.f); break;
  }
  return INV ? cconj(w) : w;
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  // 4 x 4: DFT-4 over c2 (elements c1 + 4 c2), twiddle W16^(c1 k2), DFT-4 over c1;
  // output index k2 + 4 k1.
  float2 y[16];
#pragma unroll
  for (int c1 = 0; c1 < 4; ++c1) {
    float2 a = v[c1], b = v[c1 + 4], c = v[c1 + 8], d = v[c1 + 12];
    dft4<INV>(a, b, c, d);
    y[c1 * 4 + 0] = a;
    y[c1 * 4 + 1] = (c1 == 0) ? b : cmul(b, w16<INV>(c1 * 1));
    y[c1 * 4 + 2] = (c1 == 0) ? c : (c1 == 2 ? mul_mi<INV>(c) : cmul(c, w16<INV>(c1 * 2)));
    y[c1 * 4 + 3] = (c1 == 0) ? d : cmul(d, w16<INV>(c1 * 3));
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 a = y[0 * 4 + k2], b = y[1 * 4 + k2], c = y[2 * 4 + k2], d = y[3 * 4 + k2];
    dft4<INV>(a, b, c, d);
    v[k2 + 0] = a;
    v[k2 + 4] = b;
    v[k2 + 8] = c;
    v[k2 + 12] = d;
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* u) {
  if constexpr (R == 2) {
    dft2<INV>(u[0], u[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(u[0], u[1], u[2], u[3]);
  } else if constexpr (R == 8) {
    dft8<INV>(u);
  } else {
    dft16<INV>(u);
  }
}

// --------------------------------------------------------------------- twiddle tables

// Host-side layout of the shared twiddle table of one line length: for each radix-16
// stage s with M(s) > 1, entries [(k-1) * M(s) + mu] = exp(-2 pi i mu k L(s) / PB),
// k = 1..15, mu = 0..M(s)-1; for P = 3 PB then [n] = exp(-2 pi i n / P) and
// [PB + n] = exp(-2 pi i 2n / P), n < PB.  Filled in FP64 on the host.

template <int P>
__device__ __forceinline__ void load_twiddles(float2* sm_tw, const float2* __restrict__ g_tw) {
  for (int i = threadIdx.x; i < Fft<P>::TW; i += blockDim.x) sm_tw[i] = g_tw[i];
}

// --------------------------------------------------------------------- twiddle providers

// TwTable: the per-stage table in shared memory, one load per twiddle.
struct TwTable {
  const float2* tw;
  // radix-3 twiddle W_P^{(idx / PB + 1)(idx % PB)}
  template <int P>
  __device__ __forceinline__ float2 r3(int idx) const {
    return tw[Fft<P>::TW_BASE + idx];
  }
  template <int P, int S>
  __device__ __forceinline__ float2 get(int mu, int k) const {
    return tw[Fft<P>::tw_off(S) + (k - 1) * Fft<P>::M(S) + mu];
  }
  template <int P, int S, bool INV>
  __device__ __forceinline__ void apply(float2 (&v)[16], int mu) const {
    const float2* w = tw + Fft<P>::tw_off(S) + mu;
#pragma unroll
    for (int k = 1; k < 16; ++k)
      v[k] = INV ? cmulc(v[k], w[(k - 1) * Fft<P>::M(S)]) : cmul(v[k], w[(k - 1) * Fft<P>::M(S)]);
  }
};

// TwPow: one root r = W_P^{mu L(S)} from the full table (entry k = 1), the powers r^k
// by a product tree of depth <= 4 (rounding error a few ulp), no further loads.
struct TwPow {
  const float2* tw;
  template <int P>
  __device__ __forceinline__ float2 r3(int idx) const {
    return tw[Fft<P>::TW_BASE + idx];
  }
  template <int P, int S, bool INV>
  __device__ __forceinline__ void apply(float2 (&v)[16], int mu) const {
    const float2 r = tw[Fft<P>::tw_off(S) + mu];
    pow_apply<INV>(v, r);
  }
  template <bool INV>
  __device__ __forceinline__ static void pow_apply(float2 (&v)[16], float2 r) {
    float2 w[16];
    w[1] = r;
    w[2] = cmul(r, r);
    w[3] = cmul(w[2], r);
    w[4] = cmul(w[2], w[2]);
    w[5] = cmul(w[4], r);
    w[6] = cmul(w[4], w[2]);
    w[7] = cmul(w[4], w[3]);
    w[8] = cmul(w[4], w[4]);
#pragma unroll
    for (int k = 9; k < 16; ++k) w[k] = cmul(w[8], w[k - 8]);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = INV ? cmulc(v[k], w[k]) : cmul(v[k], w[k]);
  }
};

// TwRoots: the same power tree from the compact root table (Fft<P>::ROOTS entries), which
// is small enough to keep in shared memory next to the chirp.
struct TwRoots {
  const float2* roots;
  template <int P>
  __device__ __forceinline__ float2 r3(int idx) const {
    return roots[Fft<P>::ROOTS_BASE + idx];
  }
  template <int P, int S, bool INV>
  __device__ __forceinline__ void apply(float2 (&v)[16], int mu) const {
    TwPow::pow_apply<INV>(v, roots[Fft<P>::roots_off(S) + mu]);
  }
};

// Copy the roots of every twiddled stage from the full table (block-wide).
template <int P>
__device__ __forceinline__ void load_roots(float2* sm_roots, const float2* __restrict__ g_tw) {
  using F = Fft<P>;
#pragma unroll
  for (int st = 0; st < F::N16; ++st) {
    if (F::M(st) > 1)
      for (int mu = threadIdx.x; mu < F::M(st); mu += blockDim.x)
        sm_roots[F::roots_off(st) + mu] = g_tw[F::tw_off(st) + mu];
  }
  if constexpr (F::R3)
    for (int i = threadIdx.x; i < 2 * F::PB; i += blockDim.x)
      sm_roots[F::ROOTS_BASE + i] = g_tw[F::TW_BASE + i];
}

// --------------------------------------------------------------------- stages

// Barrier over the threads of one line group: the whole block, or a named barrier
// (id >= 1) over the `count` threads of this line when several lines share a block.
struct SyncBlock {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncNamed {
  int id, count;
  __device__ __forceinline__ void operator()() const {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
  }
};

#define HOLO_SYNC() sync()

template <int P, int S, class Sync = SyncBlock, class TW = TwTable>
__device__ __forceinline__ void fwd_from(float2 (&v)[16], float2* __restrict__ sm, TW tw, int t,
                                         Sync sync = Sync()) {
  using F = Fft<P>;
  if constexpr (S < F::N16) {
    constexpr int M = F::M(S);
    constexpr bool group_in = F::HW && S == F::N16 - 1, group_out = F::HW && S == F::N16 - 2;
    if constexpr (group_in) {
      // thread 16 a + k1 takes digit d0 of (a, k1) from the rows its group wrote; no barrier
      // after the read: the only later writes to these rows come from the same threads
      const float2* hr = sm + (t >> 4) * F::HW_GROUP + F::HW_ROW * (t & 15);
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = hr[c];
    } else if constexpr (S > 0) {
      const int mu = t % M, ka = t / M;
#pragma unroll
      for (int c = 0; c < 16; ++c) v[c] = sm[spad(c * M + mu + 16 * M * ka)];
      HOLO_SYNC();
    }
    dft16<false>(v);
    if constexpr (M > 1) tw.template apply<P, S, false>(v, t % M);
    if constexpr (group_out) {
      // thread 16 a + mu holds digit k1 = k of (mu, a): row k, column mu of its group's region
      float2* hr = sm + (t >> 4) * F::HW_GROUP + (t & 15);
#pragma unroll
      for (int k = 0; k < 16; ++k) hr[F::HW_ROW * k] = v[k];
      __syncwarp();
    } else if constexpr (S < F::NST - 1) {
#pragma unroll
      for (int k = 0; k < 16; ++k) sm[spad(t + F::T * k)] = v[k];
      HOLO_SYNC();
    }
    fwd_from<P, S + 1, Sync, TW>(v, sm, tw, t, sync);
  } else if constexpr (F::RB > 0 && S == F::N16) {
    constexpr int R = F::RLAST, G = 16 / R;
#pragma unroll
    for (int g = 0; g < G; ++g) {
      float2 u[R];
      const int ka = t + F::T * g;
#pragma unroll
      for (int c = 0; c < R; ++c) u[c] = sm[spad(c + R * ka)];
      dft_small<R, false>(u);
#pragma unroll
      for (int k = 0; k < R; ++k) v[g + G * k] = u[k];
    }
    HOLO_SYNC();
  }
}

template <int P, int S, class Sync = SyncBlock, class TW = TwTable>
__device__ __forceinline__ void inv_from(float2 (&v)[16], float2* __restrict__ sm, TW tw, int t,
                                         Sync sync = Sync()) {
  using F = Fft<P>;
  if constexpr (S == F::N16) {
    if constexpr (F::RB > 0) {
      constexpr int R = F::RLAST, G = 16 / R;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        float2 u[R];
#pragma unroll
        for (int k = 0; k < R; ++k) u[k] = v[g + G * k];
        dft_small<R, true>(u);
        const int ka = t + F::T * g;
#pragma unroll
        for (int c = 0; c < R; ++c) sm[spad(c + R * ka)] = u[c];
      }
      HOLO_SYNC();
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = sm[spad(t + F::T * k)];
      HOLO_SYNC();
    }
    inv_from<P, S - 1, Sync, TW>(v, sm, tw, t, sync);
  } else if constexpr (S >= 0) {
    constexpr int M = F::M(S);
    if constexpr (M > 1) tw.template apply<P, S, true>(v, t % M);
    dft16<true>(v);
    if constexpr (F::HW && S == F::N16 - 1) {
      // adjoint of the group exchange: thread 16 a + k1 writes its row, thread 16 a + mu
      // reads column mu back
      float2* hr = sm + (t >> 4) * F::HW_GROUP;
#pragma unroll
      for (int c = 0; c < 16; ++c) hr[F::HW_ROW * (t & 15) + c] = v[c];
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = hr[F::HW_ROW * k + (t & 15)];
      inv_from<P, S - 1, Sync, TW>(v, sm, tw, t, sync);
    } else if constexpr (S > 0) {
      const int mu = t % M, ka = t / M;
      // other groups may still be reading their rows of the group exchange
      if constexpr (F::HW && S == F::N16 - 2) HOLO_SYNC();
#pragma unroll
      for (int c = 0; c < 16; ++c) sm[spad(c * M + mu + 16 * M * ka)] = v[c];
      HOLO_SYNC();
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = sm[spad(t + F::T * k)];
      HOLO_SYNC();
      inv_from<P, S - 1, Sync, TW>(v, sm, tw, t, sync);
    }
  }
}

// Radix-3 steps of P = 3 PB (see the layout notes at the top).  v[c] of thread (q, i) is
// element n + PB q (n = i + TB c) on entry to r3_split and frequency-side y_q[n] on exit;
// r3_merge is its adjoint (conjugate twiddles and roots of unity, no 1/3).
template <int P, bool INV, class Sync, class TW>
__device__ __forceinline__ void r3_butterfly_third(float2 (&v)[16], float2* __restrict__ sm, TW tw,
                                                   int t, Sync sync) {
  using F = Fft<P>;
  constexpr int PB = F::PB, TB = F::TB;
  const float h3 = 0.86602540378443865f;  // sqrt(3)/2
  const int q = t / TB, i = t % TB;
  // output q of the butterfly (x0, x1, x2): x0 + w^q x1 + w^{2q} x2 with w = W_3 (forward)
  // or conj(W_3) (inverse), i.e. x0 - (x1 + x2)/2 -/+ i sqrt(3)/2 (x1 - x2) for q = 1, 2
  const float sg = ((q == 1) != INV) ? -h3 : h3;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int n = i + TB * c;
    const float2 x0 = sm[spad(n)], x1 = sm[spad(n + PB)], x2 = sm[spad(n + 2 * PB)];
    const float2 su = cadd(x1, x2), df = csub(x1, x2);
    float2 y;
    if (q == 0) {
      y = cadd(x0, su);
    } else {
      y.x = fmaf(-0.5f, su.x, x0.x) - sg * df.y;
      y.y = fmaf(-0.5f, su.y, x0.y) + sg * df.x;
    }
    v[c] = y;
  }
  (void)tw;
  sync();
}

template <int P, class Sync, class TW>
__device__ __forceinline__ void r3_fwd(float2 (&v)[16], float2* sm, TW tw, int t, Sync sync) {
  using F = Fft<P>;
  constexpr int PB = F::PB, TB = F::TB;
  const int q = t / TB, i = t % TB;
#pragma unroll
  for (int c = 0; c < 16; ++c) sm[spad(i + TB * c + PB * q)] = v[c];
  sync();
  r3_butterfly_third<P, false>(v, sm, tw, t, sync);
  if (q > 0) {
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = cmul(v[c], tw.template r3<P>((q - 1) * PB + i + TB * c));
  }
  fwd_from<PB, 0, Sync, TW>(v, sm + q * Fft<PB>::SMEM, tw, i, sync);
}

template <int P, class Sync, class TW>
__device__ __forceinline__ void r3_inv(float2 (&v)[16], float2* sm, TW tw, int t, Sync sync) {
  using F = Fft<P>;
  constexpr int PB = F::PB, TB = F::TB;
  const int q = t / TB, i = t % TB;
  inv_from<PB, Fft<PB>::N16, Sync, TW>(v, sm + q * Fft<PB>::SMEM, tw, i, sync);
  if (q > 0) {
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = cmulc(v[c], tw.template r3<P>((q - 1) * PB + i + TB * c));
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) sm[spad(i + TB * c + PB * q)] = v[c];
  sync();
  r3_butterfly_third<P, true>(v, sm, tw, t, sync);
}

// Forward DFT (e^{-2 pi i}, unnormalised): pos layout in, fpos layout out (both strided
// natural when P is a power of two).
template <int P, class Sync, class TW>
__device__ __forceinline__ void fft_fwd_with(float2 (&v)[16], float2* sm, TW tw, int t, Sync sync) {
  if constexpr (Fft<P>::R3)
    r3_fwd<P, Sync, TW>(v, sm, tw, t, sync);
  else
    fwd_from<P, 0, Sync, TW>(v, sm, tw, t, sync);
}
template <int P>
__device__ __forceinline__ void fft_fwd(float2 (&v)[16], float2* sm, const float2* tw, int t) {
  fft_fwd_with<P, SyncBlock, TwTable>(v, sm, TwTable{tw}, t, SyncBlock());
}

// Inverse DFT without the 1/P factor (the adjoint of fft_fwd): fpos in, pos out.
template <int P, class Sync, class TW>
__device__ __forceinline__ void fft_inv_with(float2 (&v)[16], float2* sm, TW tw, int t, Sync sync) {
  if constexpr (Fft<P>::R3)
    r3_inv<P, Sync, TW>(v, sm, tw, t, sync);
  else
    inv_from<P, Fft<P>::N16, Sync, TW>(v, sm, tw, t, sync);
}
template <int P>
__device__ __forceinline__ void fft_inv(float2 (&v)[16], float2* sm, const float2* tw, int t) {
  fft_inv_with<P, SyncBlock, TwTable>(v, sm, TwTable{tw}, t, SyncBlock());
}

}  // namespace holo
