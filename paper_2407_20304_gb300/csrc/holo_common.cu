// Line-length independent kernels: pass D (grad_psi), the reductions feeding grad_q and the
// loss, FP64 inner products (Eq. DaiYuan2 coefficients) and the CG vector updates.
#include "holo.h"
#include "holo_internal.h"
#include "holo_kernels.cuh"

namespace holo {

namespace {

constexpr int kThreads = 256;

// grad_psi_k[i][ip] = 2 sum_j sum_Y wy_j(Y, i) h_kj[Y][ip]: the y-transpose of the bilinear
// resample gathered from the (at most two) box rows whose taps reach psi row i, summed
// over the distances j (Eq. gradpsi: grad = 2 sum_j L*_kj r_kj).  The rows and weights
// come from the transposed-tap table of each plane.
// One block per (psi row i, angle kl): the transposed row taps of every distance are read
// once into shared memory, then each thread sums its column pairs over j with all the
// 16-byte loads of one pair issued together.  h rows start on 16-byte boundaries (n even).
// (One psi row of one angle; the block-shared row table is filled, synchronised and read.)
__device__ __forceinline__ void pass_d_row(const PassArgs& a, int i, int kl) {
  const int n = a.n;
  __shared__ const float4* row[HOLO_MAX_DIST];
  __shared__ float w0s[HOLO_MAX_DIST], w1s[HOLO_MAX_DIST];
  if (threadIdx.x < a.J) {
    const int j = threadIdx.x;
    const long long gp = (long long)(a.k0 + kl) * a.J + j;
    const AdjTap at = a.yadj[gp * n + i];
    const PlaneDesc d = a.planes[gp];
    const float2* h = a.ybuf + (long long)(kl * a.J + j) * a.ystride;
    // rows X0 and X0 + 1 of the box; a zero weight marks a tap outside it (never read)
    int r = at.X0 - d.by0;
    float w0 = at.w0, w1 = at.w1;
    if constexpr (kBoundsCheck) {
      const bool ok = (w0 == 0.f || (r >= 0 && r < d.bys)) &&
                      (w1 == 0.f || (r + 1 >= 0 && r + 1 < d.bys)) &&
                      (long long)d.bys * n <= a.ystride;
      if (!ok) {
        flag_bounds(a.err);
        r = 0;
        w0 = w1 = 0.f;
      }
    }
    row[j] = reinterpret_cast<const float4*>(h + (long long)r * n);
    w0s[j] = w0;
    w1s[j] = w1;
  }
  __syncthreads();
  const int half = n / 2;
  float2* out = a.grad_psi + ((long long)kl * n + i) * n;
  const float2* eta = a.dy_eta ? a.dy_eta + ((long long)kl * n + i) * n : nullptr;
  float gg = 0.f, ge = 0.f;
  for (int p = threadIdx.x; p < half; p += blockDim.x) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < HOLO_MAX_DIST; ++j) {
      if (j < a.J) {
        const float w0 = w0s[j], w1 = w1s[j];
        if (w0 != 0.f) {
          const float4 z = __ldg(row[j] + p);
          acc.x = fmaf(w0, z.x, acc.x);
          acc.y = fmaf(w0, z.y, acc.y);
          acc.z = fmaf(w0, z.z, acc.z);
          acc.w = fmaf(w0, z.w, acc.w);
        }
        if (w1 != 0.f) {
          const float4 z = __ldg(row[j] + half + p);
          acc.x = fmaf(w1, z.x, acc.x);
          acc.y = fmaf(w1, z.y, acc.y);
          acc.z = fmaf(w1, z.z, acc.z);
          acc.w = fmaf(w1, z.w, acc.w);
        }
      }
    }
    float2 r0 = make_float2(2.f * acc.x, 2.f * acc.y), r1 = make_float2(2.f * acc.z, 2.f * acc.w);
    if (a.accumulate) {
      r0 = cadd(r0, out[2 * p]);
      r1 = cadd(r1, out[2 * p + 1]);
    }
    out[2 * p] = r0;
    out[2 * p + 1] = r1;
    if (a.dy_eta) {
      const float4 e = __ldg(reinterpret_cast<const float4*>(eta) + p);
      gg = fmaf(r0.x, r0.x, fmaf(r0.y, r0.y, fmaf(r1.x, r1.x, fmaf(r1.y, r1.y, gg))));
      ge = fmaf(r0.x, e.x, fmaf(r0.y, e.y, fmaf(r1.x, e.z, fmaf(r1.y, e.w, ge))));
    }
  }
  if (a.dy_eta) {
    // FP32 over the row's elements of a warp, FP64 across the warps (FP64 arithmetic is
    // scarce on this part: a block-wide FP64 reduction per row cost more than the loads)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gg += __shfl_down_sync(0xffffffffu, gg, o);
      ge += __shfl_down_sync(0xffffffffu, ge, o);
    }
    __shared__ float wsum[2][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
      wsum[0][w] = gg;
      wsum[1][w] = ge;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sgg = 0.0, sge = 0.0;
      for (int k = 0; k < nw; ++k) {
        sgg += (double)wsum[0][k];
        sge += (double)wsum[1][k];
      }
      const long long row = (long long)kl * n + i;
      a.dy_part[row] = sgg;
      a.dy_part[(long long)a.nk * n + row] = sge;
    }
  }
}

__global__ void __launch_bounds__(256) k_pass_d(const __grid_constant__ PassArgs a) {
  pass_d_row(a, blockIdx.x, blockIdx.y);
}

// Pass D of several problems in one persistent launch: items {problem, kl * n + i}.
__global__ void __launch_bounds__(256) k_pass_d_multi(const PassArgs* __restrict__ args,
                                                      const int2* __restrict__ items, int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int2 item = items[it];
    const PassArgs& a = args[item.x];
    __syncthreads();  // the previous item's row table has been read
    pass_d_row(a, item.y % a.n, item.y / a.n);
  }
}

// G'_j on the union box of the chunk: sum over angles (ascending, a fixed order) of
// conj(w_kj) v_kj.  Each thread owns kReduceEpt elements; the box descriptors of the angles
// are staged in shared memory a tile at a time, and the loads of a few angles are issued
// together (the additions stay in angle order).
constexpr int kReduceEpt = 4;
constexpr int kReduceTile = 128;
__global__ void __launch_bounds__(256) k_reduce_g(PassArgs a, float2* Gp, int j, int row0, int nrows,
                                                  int col0, int ncols, int opitch, int orow0,
                                                  int ocol0, int accumulate) {
  __shared__ int4 box[kReduceTile];
  const long long total = (long long)nrows * ncols;
  const long long base = (long long)blockIdx.x * blockDim.x * kReduceEpt + threadIdx.x;
  int Y[kReduceEpt], X[kReduceEpt];
  float2 acc[kReduceEpt];
#pragma unroll
  for (int e = 0; e < kReduceEpt; ++e) {
    const long long idx = base + (long long)e * blockDim.x;
    Y[e] = idx < total ? row0 + (int)(idx / ncols) : -(1 << 30);
    X[e] = idx < total ? col0 + (int)(idx % ncols) : -(1 << 30);
    acc[e] = make_float2(0.f, 0.f);
  }
  for (int kt = 0; kt < a.nk; kt += kReduceTile) {
    const int nt = min(kReduceTile, a.nk - kt);
    __syncthreads();
    if (threadIdx.x < nt) {
      const PlaneDesc d = a.planes[(long long)(a.k0 + kt + threadIdx.x) * a.J + j];
      box[threadIdx.x] = make_int4(d.by0, d.bys, d.bx0, d.bxs);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < nt; ++kk) {
      const int4 d = box[kk];
      const float2* gk = a.gkbuf + (long long)((kt + kk) * a.J + j) * a.gkstride;
#pragma unroll
      for (int e = 0; e < kReduceEpt; ++e) {
        const int ry = Y[e] - d.x, rx = X[e] - d.z;
        if ((unsigned)ry < (unsigned)d.y && (unsigned)rx < (unsigned)d.w)
          acc[e] = cadd(acc[e], __ldg(gk + (long long)ry * d.w + rx));
      }
    }
  }
#pragma unroll
  for (int e = 0; e < kReduceEpt; ++e) {
    const long long idx = base + (long long)e * blockDim.x;
    if (idx < total) {
      float2* o = Gp + (long long)(Y[e] - orow0) * opitch + (X[e] - ocol0);
      *o = accumulate ? cadd(*o, acc[e]) : acc[e];
    }
  }
}

// Column-blocked copy of amplitude images for pass B: out[p][gr][r][c] = in[p][r][gr C + c]
// (zero where gr C + c >= n), so the C columns of a pass-B column group are contiguous per
// row.  A block moves a tile of 32 rows x W columns (W a multiple of C) of one image through
// shared memory: the rows are read and the groups' runs of 32 x C values written contiguously.
constexpr int kBlkRows = 32;
template <int C>
__global__ void __launch_bounds__(256) k_block_data(const float* __restrict__ in, int n,
                                                    float* __restrict__ out) {
  // W = max(64, C) columns of kBlkRows rows per block; C a power of two, so the index
  // arithmetic is shifts and masks
  constexpr int W = C >= 64 ? C : 64;
  __shared__ float tile[kBlkRows][W + 1];
  const long long p = blockIdx.z;
  const int r0 = blockIdx.x * kBlkRows, c0 = blockIdx.y * W;
  const int groups = (n + C - 1) / C;
  const float* src = in + p * n * (long long)n;
  for (int e = threadIdx.x; e < kBlkRows * W; e += blockDim.x) {
    const int rr = e / W, cc = e % W, r = r0 + rr, col = c0 + cc;
    tile[rr][cc] = (r < n && col < n) ? __ldg(src + (long long)r * n + col) : 0.f;
  }
  __syncthreads();
  const int g0 = c0 / C, ng = min(W / C, groups - g0), rows = min(kBlkRows, n - r0);
  float* dst = out + (p * groups + g0) * (long long)n * C;
  for (int e = threadIdx.x; e < kBlkRows * W; e += blockDim.x) {
    const int gl = e / (kBlkRows * C), rr = (e / C) % kBlkRows, cc = e % C;
    if (gl < ng && rr < rows) dst[((long long)gl * n + r0 + rr) * C + cc] = tile[rr][gl * C + cc];
  }
}

// Reference-image term (Eq. min1, second norm): r_ref = b - a b/|b|, loss partials.
__global__ void k_ref_residual(const float2* __restrict__ b, const float* __restrict__ aref,
                               long long n2, float2* __restrict__ rref, double* part,
                               int functional) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 u = b[e];
    const float dat = aref[e];
    const float i2 = fmaf(u.x, u.x, u.y * u.y);
    float diff, s;
    if (functional) {  // F1: (|b|^2 - d_ref)^2, r = 2 (|b|^2 - d_ref) b
      diff = i2 - dat;
      s = 2.f * diff;
    } else {           // F2: (|b| - a_ref)^2, r = b - a_ref b/|b|
      const float mag = sqrtf(i2);
      diff = mag - dat;
      s = mag > 0.f ? 1.f - dat / mag : 0.f;
    }
    acc += (double)(diff * diff);
    rref[e] = cscale(u, s);
  }
  const double s = block_sum_f64(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// q[Y][X] = a[clamp(Y - lo)][clamp(X - lo)]: an n x n amplitude embedded in the P x P grid
// with its edge values repeated (the initial probe's source before D_{-zeta_0}).
__global__ void k_embed_edge(const float* __restrict__ a, int n, int P, float2* __restrict__ q) {
  const int lo = P / 2 - n / 2;
  const long long total = (long long)P * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int Y = (int)(e / P), X = (int)(e % P);
    const int i = min(max(Y - lo, 0), n - 1), j = min(max(X - lo, 0), n - 1);
    q[e] = make_float2(a[(long long)i * n + j], 0.f);
  }
}

// Hierarchical reconstruction: out = sqrt(mean of in^2 over b x b blocks), count images of
// n x n -> (n/b) x (n/b); one thread per output pixel.
__global__ void k_bin_amplitudes(const float* __restrict__ in, long long count, int n, int b,
                                 float* __restrict__ out) {
  const int m = n / b;
  const long long total = count * m * m;
  const float inv = 1.f / (float)(b * b);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long img = e / ((long long)m * m);
    const int r = (int)(e % ((long long)m * m));
    const int i = r / m, j = r % m;
    const float* src = in + img * n * n + (long long)(i * b) * n + j * b;
    float acc = 0.f;
    for (int y = 0; y < b; ++y)
      for (int x = 0; x < b; ++x) {
        const float v = src[(long long)y * n + x];
        acc = fmaf(v, v, acc);
      }
    out[e] = sqrtf(acc * inv);
  }
}

// Linear interpolation to a twice-as-dense grid: fine pixel f sits at coarse coordinate
// (f + 1/2)/2 - 1/2 (weights 3/4 and 1/4 of the two nearest coarse pixels), edges clamped;
// count complex images of N x N -> 2N x 2N.
__global__ void k_upsample2(const float2* __restrict__ in, long long count, int N,
                            float2* __restrict__ out) {
  const int M = 2 * N;
  const long long total = count * M * M;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long img = e / ((long long)M * M);
    const int r = (int)(e % ((long long)M * M));
    const int fy = r / M, fx = r % M;
    // nearest coarse pixel m = f / 2 gets 3/4; its neighbour on the side of f gets 1/4
    const int my = fy >> 1, mx = fx >> 1;
    const int ny = min(max(my + ((fy & 1) ? 1 : -1), 0), N - 1);
    const int nx = min(max(mx + ((fx & 1) ? 1 : -1), 0), N - 1);
    const float2* src = in + img * N * N;
    const float2 a = src[(long long)my * N + mx], b = src[(long long)my * N + nx];
    const float2 c = src[(long long)ny * N + mx], d = src[(long long)ny * N + nx];
    float2 v;
    v.x = 0.5625f * a.x + 0.1875f * (b.x + c.x) + 0.0625f * d.x;
    v.y = 0.5625f * a.y + 0.1875f * (b.y + c.y) + 0.0625f * d.y;
    out[e] = v;
  }
}

// Deterministic single-block sum of FP64 partials.
__global__ void k_sum_f64(const double* __restrict__ part, int count, double* out, int accumulate) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  const double s = block_sum_f64(acc, red);
  if (threadIdx.x == 0) *out = accumulate ? *out + s : s;
}

// Running loss of the context: red[3] = (acc ? red[3] : 0) + red[0] + wref red[1].
// red[0]: plane loss of the last launch group, red[1]: reference term.  red[3] is the
// running total across calls (holo_read_loss), red[7] the total of the current call.
__global__ void k_loss_total(double* red, double wref, int acc, int first) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double l = red[0] + wref * red[1];
    red[3] = (acc ? red[3] : 0.0) + l;
    red[7] = (first ? 0.0 : red[7]) + l;
  }
}

// Re <a, b> = Re sum conj(a) b: FP32 products summed in FP32 over at most 16 elements per
// thread-iteration, then FP64.
__global__ void k_dot(const float2* __restrict__ a, const float2* __restrict__ b, long long n,
                      double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  while (e < n) {
    float s = 0.f;
#pragma unroll 4
    for (int r = 0; r < 16 && e < n; ++r, e += stride) {
      const float2 x = a[e], y = b[e];
      s = fmaf(x.x, y.x, fmaf(x.y, y.y, s));
    }
    acc += (double)s;
  }
  const double s = block_sum_f64(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// The three inner products of the Dai-Yuan coefficient in one pass: Re<g, g>, Re<g, eta>,
// Re<g_prev, eta>, with the grouping of k_dot (FP32 over 16 elements, then FP64).  Partial
// sums of block b go to part[b], part[nb + b], part[2 nb + b].
__global__ void k_dot3(const float2* __restrict__ g, const float2* __restrict__ gp,
                       const float2* __restrict__ eta, long long n, double* part) {
  __shared__ double red[32];
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  while (e < n) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
    for (int r = 0; r < 16 && e < n; ++r, e += stride) {
      const float2 x = g[e], y = gp[e], d = eta[e];
      s0 = fmaf(x.x, x.x, fmaf(x.y, x.y, s0));
      s1 = fmaf(x.x, d.x, fmaf(x.y, d.y, s1));
      s2 = fmaf(y.x, d.x, fmaf(y.y, d.y, s2));
    }
    a0 += (double)s0;
    a1 += (double)s1;
    a2 += (double)s2;
  }
  const double r0 = block_sum_f64(a0, red);
  const double r1 = block_sum_f64(a1, red);
  const double r2 = block_sum_f64(a2, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = r0;
    part[gridDim.x + blockIdx.x] = r1;
    part[2 * gridDim.x + blockIdx.x] = r2;
  }
}

// eta = -g + beta eta, then x += gamma eta (the new eta): holo_direction then holo_step.
__global__ void k_direction_step(float2* __restrict__ x, float2* __restrict__ eta,
                                 const float2* __restrict__ g, float beta, float gamma, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 a = eta[e], d = g[e], xo = x[e];
    const float2 en = make_float2(fmaf(beta, a.x, -d.x), fmaf(beta, a.y, -d.y));
    eta[e] = en;
    x[e] = make_float2(fmaf(gamma, en.x, xo.x), fmaf(gamma, en.y, xo.y));
  }
}

// k_direction_step with Re <g, eta_new> accumulated as holo_dot accumulates (FP32 over 16
// elements of a thread, then FP64), one partial per block.
__global__ void k_direction_step_dot(float2* __restrict__ x, float2* __restrict__ eta,
                                     const float2* __restrict__ g, float beta, float gamma,
                                     long long n, double* __restrict__ part) {
  __shared__ double red[32];
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double acc = 0.0;
  while (e < n) {
    float s = 0.f;
    for (int r = 0; r < 16 && e < n; ++r, e += stride) {
      const float2 a = eta[e], d = g[e], xo = x[e];
      const float2 en = make_float2(fmaf(beta, a.x, -d.x), fmaf(beta, a.y, -d.y));
      eta[e] = en;
      x[e] = make_float2(fmaf(gamma, en.x, xo.x), fmaf(gamma, en.y, xo.y));
      s = fmaf(d.x, en.x, fmaf(d.y, en.y, s));
    }
    acc += (double)s;
  }
  const double t = block_sum_f64(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_axpy(float2* __restrict__ x, const float2* __restrict__ eta, float gamma,
                       long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 a = x[e], d = eta[e];
    x[e] = make_float2(fmaf(gamma, d.x, a.x), fmaf(gamma, d.y, a.y));
  }
}

__global__ void k_direction(float2* __restrict__ eta, const float2* __restrict__ g, float beta,
                            long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 a = eta[e], d = g[e];
    eta[e] = make_float2(fmaf(beta, a.x, -d.x), fmaf(beta, a.y, -d.y));
  }
}

__global__ void k_scale_add(float2* __restrict__ out, const float2* __restrict__ in, float alpha,
                            long long n, int accumulate) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    float2 r = cscale(in[e], alpha);
    if (accumulate) r = cadd(r, out[e]);
    out[e] = r;
  }
}

__global__ void k_fill_zero(float2* __restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = make_float2(0.f, 0.f);
}

int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_pass_d(const PassArgs& a, cudaStream_t s) {
  dim3 grid(a.n, a.nk);
  k_pass_d<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pass_d_multi(const PassArgs* args, const int2* items, int nitems, int nblocks,
                                cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_pass_d_multi<<<nblocks < nitems ? nblocks : nitems, 256, 0, s>>>(args, items, nitems);
  return cudaGetLastError();
}

cudaError_t launch_reduce_g(const PassArgs& a, float2* out, int j, int row0, int nrows, int col0,
                            int ncols, int opitch, int orow0, int ocol0, int accumulate,
                            cudaStream_t s) {
  const long long total = (long long)nrows * ncols;
  if (total <= 0) return cudaSuccess;
  const long long per = 256LL * kReduceEpt;
  k_reduce_g<<<(unsigned)((total + per - 1) / per), 256, 0, s>>>(a, out, j, row0, nrows, col0,
                                                                 ncols, opitch, orow0, ocol0,
                                                                 accumulate);
  return cudaGetLastError();
}

cudaError_t launch_ref_residual(const float2* bref, const float* sqrt_dref, long long n2,
                                float2* rref, double* part, int nblocks, int functional,
                                cudaStream_t s) {
  k_ref_residual<<<nblocks, kThreads, 0, s>>>(bref, sqrt_dref, n2, rref, part, functional);
  return cudaGetLastError();
}

cudaError_t launch_embed_edge(const float* a, int n, int P, float2* q, cudaStream_t s) {
  k_embed_edge<<<grid_for((long long)P * P), kThreads, 0, s>>>(a, n, P, q);
  return cudaGetLastError();
}

cudaError_t launch_block_data(const float* in, long long planes, int n, int C, float* out,
                              cudaStream_t s) {
  if (planes <= 0) return cudaSuccess;
  const int W = C >= 64 ? C : 64;  // a multiple of C (C is a power of two, 2 .. 256)
  const int groups = (n + C - 1) / C;
  const dim3 grid((n + kBlkRows - 1) / kBlkRows, (groups * C + W - 1) / W, (unsigned)planes);
  switch (C) {
    case 2: k_block_data<2><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 4: k_block_data<4><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 8: k_block_data<8><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 16: k_block_data<16><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 32: k_block_data<32><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 64: k_block_data<64><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 128: k_block_data<128><<<grid, kThreads, 0, s>>>(in, n, out); break;
    case 256: k_block_data<256><<<grid, kThreads, 0, s>>>(in, n, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bin_amplitudes(const float* in, long long count, int n, int b, float* out,
                                  cudaStream_t s) {
  const long long total = count * (n / b) * (long long)(n / b);
  if (total <= 0) return cudaSuccess;
  k_bin_amplitudes<<<grid_for(total), kThreads, 0, s>>>(in, count, n, b, out);
  return cudaGetLastError();
}

cudaError_t launch_upsample2(const float2* in, long long count, int N, float2* out,
                             cudaStream_t s) {
  const long long total = count * 4LL * N * N;
  if (total <= 0) return cudaSuccess;
  k_upsample2<<<grid_for(total), kThreads, 0, s>>>(in, count, N, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double* part, int count, double* out, int accumulate,
                           cudaStream_t s) {
  k_sum_f64<<<1, 1024, 0, s>>>(part, count, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_loss_total(double* red, double wref, int acc, int first, cudaStream_t s) {
  k_loss_total<<<1, 32, 0, s>>>(red, wref, acc, first);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float2* a, const float2* b, long long n, double* part, int nblocks,
                       cudaStream_t s) {
  k_dot<<<nblocks, kThreads, 0, s>>>(a, b, n, part);
  return cudaGetLastError();
}

cudaError_t launch_dot3(const float2* g, const float2* gp, const float2* eta, long long n,
                        double* part, int nblocks, cudaStream_t s) {
  k_dot3<<<nblocks, kThreads, 0, s>>>(g, gp, eta, n, part);
  return cudaGetLastError();
}

cudaError_t launch_direction_step_dot(float2* x, float2* eta, const float2* g, float beta,
                                      float gamma, long long n, double* part, int* nblocks,
                                      cudaStream_t s) {
  *nblocks = grid_for(n);
  k_direction_step_dot<<<*nblocks, kThreads, 0, s>>>(x, eta, g, beta, gamma, n, part);
  return cudaGetLastError();
}

cudaError_t launch_direction_step(float2* x, float2* eta, const float2* g, float beta, float gamma,
                                  long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_direction_step<<<grid_for(n), kThreads, 0, s>>>(x, eta, g, beta, gamma, n);
  return cudaGetLastError();
}

cudaError_t launch_axpy(float2* x, const float2* eta, float gamma, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_axpy<<<grid_for(n), kThreads, 0, s>>>(x, eta, gamma, n);
  return cudaGetLastError();
}

cudaError_t launch_direction(float2* eta, const float2* g, float beta, long long n,
                             cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_direction<<<grid_for(n), kThreads, 0, s>>>(eta, g, beta, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_add(float2* out, const float2* in, float alpha, long long n,
                             int accumulate, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scale_add<<<grid_for(n), kThreads, 0, s>>>(out, in, alpha, n, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_fill_zero(float2* out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill_zero<<<grid_for(n), kThreads, 0, s>>>(out, n);
  return cudaGetLastError();
}

}  // namespace holo
