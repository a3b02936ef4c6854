// Line-length independent kernels: pass D (grad_psi), the reductions feeding grad_q and the
// loss, FP64 inner products (Eq. DaiYuan2 coefficients) and the CG vector updates.
#include "holo_internal.h"
#include "holo_kernels.cuh"

namespace holo {

namespace {

constexpr int kThreads = 256;

// grad_psi_k[i][ip] = 2 sum_j sum_Y wy_j(Y, i) h_kj[Y][ip]: the y-transpose of the bilinear
// resample gathered from the (at most two) box rows whose taps reach psi row i, summed
// over the distances j (Eq. gradpsi: grad = 2 sum_j L*_kj r_kj).  The rows and weights
// come from the transposed-tap table of each plane.
__global__ void k_pass_d(PassArgs a) {
  const int n = a.n, i = blockIdx.x, kl = blockIdx.y;
  float2* out = a.grad_psi + ((long long)kl * n + i) * n;
  for (int ip = threadIdx.x; ip < n; ip += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int j = 0; j < a.J; ++j) {
      const long long gp = (long long)(a.k0 + kl) * a.J + j;
      const AdjTap at = a.yadj[gp * n + i];
      const PlaneDesc d = a.planes[gp];
      const float2* h = a.ybuf + (long long)(kl * a.J + j) * a.ystride;
      const int r0 = at.X0 - d.by0;
      if (at.w0 != 0.f) {
        const float2 z = h[(long long)r0 * n + ip];
        acc.x = fmaf(at.w0, z.x, acc.x);
        acc.y = fmaf(at.w0, z.y, acc.y);
      }
      if (at.w1 != 0.f) {
        const float2 z = h[(long long)(r0 + 1) * n + ip];
        acc.x = fmaf(at.w1, z.x, acc.x);
        acc.y = fmaf(at.w1, z.y, acc.y);
      }
    }
    float2 r = make_float2(2.f * acc.x, 2.f * acc.y);
    if (a.accumulate) r = cadd(r, out[ip]);
    out[ip] = r;
  }
}

// G'_j on the union box of the chunk: sum over angles (fixed order) of conj(w_kj) v_kj.
__global__ void k_reduce_g(PassArgs a, float2* Gp, int j, int row0, int nrows, int col0,
                           int ncols) {
  const long long total = (long long)nrows * ncols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int Y = row0 + (int)(idx / ncols), X = col0 + (int)(idx % ncols);
    float2 acc = make_float2(0.f, 0.f);
    for (int kl = 0; kl < a.nk; ++kl) {
      const PlaneDesc d = a.planes[(long long)(a.k0 + kl) * a.J + j];
      const int ry = Y - d.by0, rx = X - d.bx0;
      if ((unsigned)ry < (unsigned)d.bys && (unsigned)rx < (unsigned)d.bxs)
        acc = cadd(acc, a.gkbuf[(long long)(kl * a.J + j) * a.gkstride + (long long)ry * d.bxs + rx]);
    }
    Gp[idx] = acc;
  }
}

// Reference-image term (Eq. min1, second norm): r_ref = b - a b/|b|, loss partials.
__global__ void k_ref_residual(const float2* __restrict__ b, const float* __restrict__ aref,
                               long long n2, float2* __restrict__ rref, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 u = b[e];
    const float amp = aref[e];
    const float mag = sqrtf(fmaf(u.x, u.x, u.y * u.y));
    const float diff = mag - amp;
    acc += (double)(diff * diff);
    const float s = mag > 0.f ? 1.f - amp / mag : 0.f;
    rref[e] = cscale(u, s);
  }
  const double s = block_sum_f64(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
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
__global__ void k_loss_total(double* red, double wref, int acc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) red[3] = (acc ? red[3] : 0.0) + red[0] + wref * red[1];
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
  k_pass_d<<<grid, a.n >= 1024 ? 512 : kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce_g(const PassArgs& a, float2* Gp, int j, int row0, int nrows, int col0,
                            int ncols, cudaStream_t s) {
  const long long total = (long long)nrows * ncols;
  if (total <= 0) return cudaSuccess;
  k_reduce_g<<<grid_for(total), kThreads, 0, s>>>(a, Gp, j, row0, nrows, col0, ncols);
  return cudaGetLastError();
}

cudaError_t launch_ref_residual(const float2* bref, const float* sqrt_dref, long long n2,
                                float2* rref, double* part, int nblocks, cudaStream_t s) {
  k_ref_residual<<<nblocks, kThreads, 0, s>>>(bref, sqrt_dref, n2, rref, part);
  return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double* part, int count, double* out, int accumulate,
                           cudaStream_t s) {
  k_sum_f64<<<1, 1024, 0, s>>>(part, count, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_loss_total(double* red, double wref, int acc, cudaStream_t s) {
  k_loss_total<<<1, 32, 0, s>>>(red, wref, acc);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float2* a, const float2* b, long long n, double* part, int nblocks,
                       cudaStream_t s) {
  k_dot<<<nblocks, kThreads, 0, s>>>(a, b, n, part);
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
