// holo_dot_noalloc: the FP64 inner product Re <a, b> without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need an inner product:
// code that runs while a memory pool or another runtime owns all free memory, callers
// inside allocation-free regions of a larger application (e.g. between a planner's
// fixed budget and its launch), or embedders that forbid the library from calling
// cudaMalloc at all.  holo_dot allocates its partial sums in a context; this entry point
// keeps them in a file-scope device array instead, so it needs no context and makes no
// allocation.  The caller passes the two input arrays and a host output scalar.
//
// Scratch: g_dot_scratch holds one FP64 partial per block of kElemsPerBlock elements plus
// the final sum, kScratchDoubles + 1 doubles (512 KiB + 8 B) in every GPU that loads the
// library, until the process exits.  Inputs longer than kScratchDoubles * kElemsPerBlock
// elements are rejected with HOLO_ERR_UNSUPPORTED before any device work.
//
// The array's name in host code is a host-side stand-in, not a device address: its device
// address is obtained once per device with cudaGetSymbolAddress (on the first call made on
// that device, with that device current) and passed to the kernels.  Every call writes all
// the partials it later reads, so nothing has to be cleared between calls; calls that
// overlap on the GPU (e.g. on two streams) share the array and race.
#include <mutex>

#include "holo.h"
#include "holo_kernels.cuh"

namespace {

constexpr int kScratchDoubles = 65536;
constexpr int kElemsPerBlock = 4096;   // 256 threads x 16 elements
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dot_scratch[kScratchDoubles + 1];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Per-block partial of Re sum conj(a) b over elements [blockIdx.x * 4096, +4096):
// 16 FP32 products per thread summed in FP32, then the block in FP64.
__global__ void k_dot_partials(const float2* __restrict__ a, const float2* __restrict__ b,
                               long long n, double* __restrict__ part) {
  __shared__ double red[32];
  const long long base = (long long)blockIdx.x * kElemsPerBlock + threadIdx.x;
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < kElemsPerBlock / kThreads; ++r) {
    const long long e = base + (long long)r * kThreads;
    if (e < n) {
      const float2 x = a[e], y = b[e];
      s = fmaf(x.x, y.x, fmaf(x.y, y.y, s));
    }
  }
  const double t = holo::block_sum_f64((double)s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_dot_final(const double* __restrict__ part, int count, double* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  const double t = holo::block_sum_f64(acc, red);
  if (threadIdx.x == 0) *out = t;
}

// True when p is device (or managed) memory that kernels on device `dev` may read.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// Device address of g_dot_scratch on the current device (set up once per device).
holo_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HOLO_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dot_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HOLO_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)p;
  }
  *out = g_scratch_ptr[dev];
  return HOLO_OK;
}

}  // namespace

extern "C" holo_status holo_dot_noalloc(const void* a, const void* b, long long n_c64,
                                        double* re_out, void* stream) {
  if (!a || !b || !re_out || n_c64 < 0) return HOLO_ERR_ARG;
  if (n_c64 > (long long)kScratchDoubles * kElemsPerBlock) return HOLO_ERR_UNSUPPORTED;
  // both inputs must live on the current device, whose copy of the scratch array the kernels
  // use (checked before any device work)
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HOLO_ERR_CUDA;
  }
  if (!on_device(a, dev) || !on_device(b, dev)) return HOLO_ERR_ARG;
  double* scratch = nullptr;
  holo_status st = scratch_for_current_device(&scratch);
  if (st != HOLO_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)((n_c64 + kElemsPerBlock - 1) / kElemsPerBlock);
  if (nb > 0) {
    k_dot_partials<<<nb, kThreads, 0, s>>>((const float2*)a, (const float2*)b, n_c64, scratch);
    if (cudaGetLastError() != cudaSuccess) return HOLO_ERR_CUDA;
  }
  k_dot_final<<<1, 1024, 0, s>>>(scratch, nb, scratch + kScratchDoubles);
  if (cudaGetLastError() != cudaSuccess) return HOLO_ERR_CUDA;
  if (cudaMemcpyAsync(re_out, scratch + kScratchDoubles, sizeof(double), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HOLO_ERR_CUDA;
  }
  return HOLO_OK;
}
