// C ABI of the holography functional library (declared in include/holo.h).
//
// Host side: argument validation, FP64 geometry and tables, per-plane resample boxes,
// workspace management, and the launch sequence of one forward / gradient evaluation.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda.h>

#include "holo.h"
#include "holo_internal.h"

namespace holo {
const Ops* ops_16();
const Ops* ops_32();
const Ops* ops_64();
const Ops* ops_128();
const Ops* ops_256();
const Ops* ops_512();
const Ops* ops_1024();
const Ops* ops_2048();
const Ops* ops_4096();
const Ops* ops_48();
const Ops* ops_96();
const Ops* ops_192();
const Ops* ops_384();
const Ops* ops_768();
const Ops* ops_1536();
const Ops* ops_3072();

const Ops* ops_for(int P) {
  switch (P) {
    case 16: return ops_16();
    case 32: return ops_32();
    case 64: return ops_64();
    case 128: return ops_128();
    case 256: return ops_256();
    case 512: return ops_512();
    case 1024: return ops_1024();
    case 2048: return ops_2048();
    case 4096: return ops_4096();
    case 48: return ops_48();
    case 96: return ops_96();
    case 192: return ops_192();
    case 384: return ops_384();
    case 768: return ops_768();
    case 1536: return ops_1536();
    case 3072: return ops_3072();
    default: return nullptr;
  }
}
}  // namespace holo

using holo::LineArgs;
using holo::PassArgs;
using holo::PlaneDesc;

// holo_gradient_host splits a chunk of at least 2 kHostMinPart angles into at most
// kHostParts parts so that host<->device copies of one part overlap the planes of another.
// Part sizes follow kHostWeights: a small first part (the copy nothing hides) and a small
// last part (the result copy nothing hides).
constexpr int kHostParts = 8;
constexpr int kHostMinPart = 2;
constexpr int kHostWeights[kHostParts] = {1, 2, 3, 3, 3, 3, 3, 2};

// d_red: kRed doubles; word kErrWord holds the device-wait error flag (as 64-bit integer).
constexpr int kRed = 13;
// d_red[10 .. 12]: the Dai-Yuan inner products formed inside holo_gradient (pass D) and
// holo_direction_step_dy, read by holo_read_dy
constexpr int kDyWord = 10;
constexpr int kErrWord = 8;

struct holo_ctx {
  holo_geometry geo{};
  int n = 0, P = 0, J = 0, K = 0, chunk = 0;
  float ext = 1.f;
  double wref = 0.0;
  int functional = HOLO_F2_AMPLITUDE;
  // schedule (holo_set_schedule): row-pass blocks per SM (0: as many as fit), pass-B Y stage
  // and plane-split form (-1: automatic, 0: off, 1: on where applicable)
  int sched_row_per_sm = 0, sched_stage = -1, sched_split = -1;
  cudaStream_t stream = nullptr;
  // holo_gradient_host in parts: copy streams and their events (created on first use)
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  cudaEvent_t ev_start = nullptr, ev_out = nullptr, ev_q = nullptr;
  cudaEvent_t ev_in[kHostParts] = {}, ev_done[kHostParts] = {};
  const holo::Ops* ops = nullptr;
  double mt[HOLO_MAX_DIST] = {}, omega[HOLO_MAX_DIST] = {}, zeta[HOLO_MAX_DIST] = {},
         zhat[HOLO_MAX_DIST] = {};
  // tables
  float2* d_tw = nullptr;
  float2* d_chirp_zhat = nullptr;   // [J][P]
  float2* d_chirp_omega = nullptr;  // [J][P]
  float2* d_chirp_zeta0 = nullptr;  // [P]
  float2* d_chirp_tmp = nullptr;    // [P]
  // planes
  std::vector<PlaneDesc> planes;
  PlaneDesc* d_planes = nullptr;
  bool have_shifts = false;
  std::vector<float> t_host;       // sample shifts t [K][J][2] as given
  // probe shifts s [K][J][2] (holo_set_probe_shifts): the planes then use the full-grid box,
  // object shifts t - m~_j s and the per-plane phase ramps below
  bool probe_shift = false;
  std::vector<float> s_host;
  float2* d_ramp_x = nullptr;      // [K * J][P]: exp(-2 pi i k s_x / P)
  float2* d_ramp_y = nullptr;      // [K * J][P]: exp(-2 pi i k s_y / P)
  size_t ramp_bytes = 0;
  int maxbys = 0, maxbxs = 0;
  // FP64-built bilinear tap tables and the flat row list of all planes
  holo::Tap* d_xtap = nullptr;
  holo::Tap* d_ytap = nullptr;
  holo::AdjTap* d_xadj = nullptr;
  holo::AdjTap* d_yadj = nullptr;
  int2* d_lines = nullptr;      // line -> {plane, box row}
  std::vector<int> rowstart;    // first line of each plane (host)
  int tap_stride = 0;
  size_t tap_bytes = 0;
  // data: the amplitudes of holo_set_data copied into pass B's column-blocked layout
  // [n_angles][J][groups][n][C]; the reference image is used in place
  float* d_dblk = nullptr;
  size_t dblk_bytes = 0;
  const float* sqrt_dref = nullptr;
  bool have_data = false;
  // probe
  float2* d_pj = nullptr;  // [J][P][P]
  float2* d_b = nullptr;   // [n][n]
  bool have_probe = false;
  // per-plane workspace
  float2* ybuf = nullptr;
  long long ystride = 0;
  float2* gkbuf = nullptr;
  long long gkstride = 0;
  size_t ws_bytes_planes = 0;
  // evaluation scratch
  float2* d_scratch = nullptr;  // P*P
  // holo_set_dy_direction: the direction eta whose Dai-Yuan products pass D forms, and the
  // FP64 partials of those products (pass D rows, direction-step blocks)
  const float2* dy_eta = nullptr;
  double* d_dypart = nullptr;
  size_t dypart_bytes = 0;
  // row stages of the probe-gradient sources, [sum of their rows][P] (eval_qfinish)
  float2* d_qscr = nullptr;
  size_t qscr_bytes = 0;
  float2* d_T = nullptr;        // n*n
  // deferred probe gradient (HOLO_DEFER_Q): per distance the union box {row0, rows, col0, cols}
  // of every plane's box, and G'_j accumulated on it (offset gacc_off[j] in d_gacc)
  int qbox[HOLO_MAX_DIST][4] = {};
  float2* d_gacc = nullptr;
  size_t gacc_bytes = 0;
  size_t gacc_off[HOLO_MAX_DIST] = {};
  bool q_pending = false;
  float2* d_rref = nullptr;     // n*n
  double* d_part = nullptr;
  long long part_cap = 0;
  double* d_dot3 = nullptr;     // partial sums of holo_dy_dots: 3 x (8 x SM count)
  float2* d_tpart = nullptr;    // pass B (plane-split form): partial residual sums
  size_t tpart_bytes = 0;
  double* d_red = nullptr;      // kRed doubles: loss, reference term, dot, running loss, DY
                                // dots, call loss; word kErrWord: device-wait error flag
  double* h_red = nullptr;      // pinned, kRed doubles
  // pass B's Y stage: TMA tensor map over ybuf (device, 128 bytes), used when ystage
  void* d_ymap = nullptr;
  bool ystage = false;
  // host-buffer staging
  float2* s_psi = nullptr;
  float2* s_gpsi = nullptr;
  float* s_data = nullptr;
  float* s_dblk = nullptr;      // the chunk's data of the host call, column-blocked
  float2* s_q = nullptr;
  float2* s_gq = nullptr;
  long long bytes = 0;
  long long launches = 0;
  std::string err;
  // per-pass event timing
  bool timing = false;
  struct Rec {
    int id;
    cudaEvent_t a, b;
    long long launches;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

namespace {

constexpr int kRefBlocks = 64;

holo_status fail(holo_ctx* c, holo_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define HOLO_CK(ctx, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail((ctx), HOLO_ERR_CUDA,                                                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

#define HOLO_LAUNCH(ctx, call)   \
  do {                           \
    HOLO_CK(ctx, call);          \
    (ctx)->launches++;           \
  } while (0)

// Host-side fault injection for tests (nothing faults on the GPU): the environment variable
// HOLO_FAULT holds a comma-separated list of kinds, read at every check.
//   alloc  every workspace allocation fails (HOLO_ERR_OOM) before cudaMalloc is called;
//   arg    every forward / gradient call is rejected as an invalid argument (HOLO_ERR_ARG)
//          before any device work;
//   nan    every loss read reports a non-finite loss (HOLO_ERR_NUMERIC).
bool fault_on(const char* kind) {
  const char* e = std::getenv("HOLO_FAULT");
  if (!e || !*e) return false;
  const std::string list = std::string(",") + e + ",";
  return list.find(std::string(",") + kind + ",") != std::string::npos;
}

holo_status dalloc(holo_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HOLO_OK;
  if (fault_on("alloc"))
    return fail(c, HOLO_ERR_OOM, "allocation failure injected by HOLO_FAULT=alloc");
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? HOLO_ERR_OOM : HOLO_ERR_CUDA,
                std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  c->bytes += (long long)bytes;
  return HOLO_OK;
}

void dfree(holo_ctx* c, void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    c->bytes -= (long long)bytes;
  }
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Pass B's Y stage: a TMA tensor map over ybuf viewed as a row-major [planes * maxbys][2n]
// float matrix, boxes of 2C floats x kStageBox rows.  Used only where the driver provides
// the encoder, n is even (16-byte row pitch) and the stage leaves pass B's resident blocks
// per SM unchanged; otherwise pass B loads Y directly.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

holo_status encode_ystage(holo_ctx* c, int maxbys) {
  c->ystage = false;
  const int n = c->n, C = c->ops->pass_b_cols;
  if (n % 2 || !c->ops->pass_b_stage_ok(n, maxbys)) return HOLO_OK;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return HOLO_OK;
  const long long rows = (long long)c->chunk * c->J * (c->ystride / n);
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * n, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * C), (cuuint32_t)holo::kStageBox};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->ybuf, dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return HOLO_OK;
  HOLO_CK(c, cudaMemcpyAsync(c->d_ymap, &m, sizeof(m), cudaMemcpyHostToDevice, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  c->ystage = true;
  return HOLO_OK;
}

// Scoped event pair around a group of launches of one pass (no-op unless timing is on).
// NVTX range names of the pass ids (HOLO_T_*), seen by nsys / ncu --nvtx
constexpr const char* kPassRange[HOLO_NUM_TIMERS] = {
    "holo:probe", "holo:pass_a", "holo:pass_b", "holo:pass_c",
    "holo:pass_d", "holo:qgrad",  "holo:reduce", "holo:vector"};

// Per-pass scope: an NVTX range around the pass's launches (always; the calls cost a pointer
// test when no tool is attached) and, while timing is on, CUDA events on the context's stream.
struct PassTimer {
  holo_ctx* c;
  int id;
  long long l0;
  cudaEvent_t a = nullptr;
  PassTimer(holo_ctx* ctx, int pass) : c(ctx), id(pass), l0(ctx->launches) {
    nvtxRangePushA(kPassRange[pass]);
    if (!c->timing) return;
    a = take();
    if (a) cudaEventRecord(a, c->stream);
  }
  cudaEvent_t take() {
    if (!c->pool.empty()) {
      cudaEvent_t e = c->pool.back();
      c->pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  ~PassTimer() {
    nvtxRangePop();
    if (!c->timing || !a) return;
    cudaEvent_t b = take();
    if (!b) return;
    cudaEventRecord(b, c->stream);
    c->recs.push_back({id, a, b, c->launches - l0});
  }
};


// exp(-i pi lambda z f^2) / P with f = k/(P dx), k in [-P/2, P/2)  (reading of D_z), FP64.
std::vector<float2> chirp_table(int P, double lambda, double dx, double z) {
  std::vector<float2> c(P);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < P; ++k) {
    const double kk = k < P / 2 ? k : k - P;
    const double f = kk / (P * dx);
    const double ph = -pi * lambda * z * f * f;
    c[k] = make_float2((float)(std::cos(ph) / P), (float)(std::sin(ph) / P));
  }
  return c;
}

// Twiddle table in the layout of holo_fft.cuh for P = PB or 3 PB (PB a power of two):
// radix-16 stage s with M(s) = PB/16^(s+1) > 1 contributes entries
// [(k-1) M + mu] = exp(-2 pi i mu k 16^s / PB), k = 1..15; for P = 3 PB the radix-3 step
// adds exp(-2 pi i r n / P) for r = 1, 2 (outer) and n < PB (inner).
std::vector<float2> twiddle_table(int P) {
  std::vector<float2> tw;
  const int PB = P % 3 == 0 ? P / 3 : P;
  int log2p = 0;
  while ((1 << log2p) < PB) ++log2p;
  const int n16 = log2p / 4;
  const double pi = 3.14159265358979323846;
  long long L = 1;
  for (int s = 0; s < n16; ++s) {
    const long long M = PB / (L * 16);
    if (M > 1)
      for (int k = 1; k < 16; ++k)
        for (long long mu = 0; mu < M; ++mu) {
          const double a = -2.0 * pi * (double)(mu * k * L) / PB;
          tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
        }
    L *= 16;
  }
  if (PB != P)
    for (int r = 1; r <= 2; ++r)
      for (int nn = 0; nn < PB; ++nn) {
        const double a = -2.0 * pi * (double)(r * nn) / P;
        tw.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
      }
  return tw;
}

// Line lengths with kernels: 2^k (16 .. 4096) and 3 * 2^k (48 .. 3072).
bool supported_line(int P) {
  const int PB = P % 3 == 0 ? P / 3 : P;
  return is_pow2(PB) && PB >= 16 && P <= 4096;
}

// m~ = hi + lo with hi holding 24 - bits significant bits, so that hi * x is exact in FP32
// for |x| < 2^bits.
void split_mt(double mt, int P, float* hi, float* lo) {
  int bits = 0;
  while ((1 << bits) <= P / 2) ++bits;
  const int sig = 24 - bits;
  int e;
  std::frexp(mt, &e);  // mt = f * 2^e, f in [0.5, 1)
  const double scale = std::ldexp(1.0, sig - e);
  const double h = std::nearbyint(mt * scale) / scale;
  *hi = (float)h;
  *lo = (float)(mt - h);
}

// Bounding box on the P-grid of the positions whose bilinear taps can reach psi's domain:
// xi = m~ (X - P/2) - t + n/2 in (-1, n), widened by one pixel each side.
void axis_box(double mt, double t, int n, int P, int* lo, int* len) {
  const double a = P / 2 + (t - n / 2 - 1.0) / mt;
  const double b = P / 2 + (t + n / 2) / mt;
  int s = (int)std::floor(a) - 1, e = (int)std::ceil(b) + 2;
  s = std::max(s, 0);
  e = std::min(e, P);
  *lo = s;
  *len = std::max(e - s, 0);
}

// Bilinear taps of the P-grid positions [lo, lo + len) along one axis (reading R4, FP64):
// xi = m~ (X - P/2) - t + n/2, i0 = floor(xi), f = xi - i0; and their transpose: for each
// psi index, the (at most two, consecutive) positions that reach it and their weights.
void axis_taps(double mt, double t, int n, int P, int lo, int len, holo::Tap* taps,
               holo::AdjTap* adj) {
  for (int i = 0; i < n; ++i) adj[i] = holo::AdjTap{0, 0.f, 0.f, 0};
  std::vector<char> seen(n, 0);
  auto add = [&](int ip, int X, double w) {
    if (ip < 0 || ip >= n || w == 0.0) return;
    holo::AdjTap& a = adj[ip];
    if (!seen[ip]) {
      seen[ip] = 1;
      a.X0 = X;
      a.w0 = (float)w;
    } else if (X == a.X0 + 1) {
      a.w1 = (float)w;
    } else if (X == a.X0) {
      a.w0 = (float)(a.w0 + w);
    }
  };
  for (int r = 0; r < len; ++r) {
    const int X = lo + r;
    const double xi = mt * (double)(X - P / 2) - t + (double)(n / 2);
    const double i0 = std::floor(xi);
    const double f = xi - i0;
    taps[r] = holo::Tap{(int)i0, (float)f};
    add((int)i0, X, 1.0 - f);
    add((int)i0 + 1, X, f);
  }
}

holo_status upload(holo_ctx* c, void* dst, const void* src, size_t bytes) {
  HOLO_CK(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  return HOLO_OK;
}

LineArgs line_args() {
  LineArgs a;
  std::memset(&a, 0, sizeof(a));
  a.alpha = 1.f;
  return a;
}

// 2D D_z of a field given as `rows` rows of width `w` occupying P-grid rows
// [r_lo, r_lo + rows) and columns [c_lo, c_lo + w); the result keeps P-grid rows
// [or_lo, or_lo + orows) and columns [oc_lo, oc_lo + ocols), written densely with row
// pitch ocols, as out = alpha D(in) (+ out when accumulate).  Rows first, then columns.
holo_status dstep2d(holo_ctx* c, const float2* in, int r_lo, int rows, int c_lo, int w,
                    float2* out, int or_lo, int orows, int oc_lo, int ocols, const float2* chirp,
                    int conj, float alpha, int accumulate) {
  const int P = c->P;
  LineArgs a = line_args();
  a.in = in;
  a.in_line_stride = w;
  a.in_step = 1;
  a.in_lo = c_lo;
  a.in_len = w;
  a.out = c->d_scratch;  // [rows][ocols]
  a.out_line_stride = ocols;
  a.out_step = 1;
  a.out_lo = oc_lo;
  a.out_len = ocols;
  a.nlines = rows;
  a.chirp = chirp;
  a.conj_chirp = conj;
  HOLO_LAUNCH(c, c->ops->rows(a, c->d_tw, c->stream));
  LineArgs b = line_args();
  b.in = c->d_scratch;
  b.in_line_stride = 1;
  b.in_step = ocols;
  b.in_lo = r_lo;
  b.in_len = rows;
  b.out = out;
  b.out_line_stride = 1;
  b.out_step = ocols;
  b.out_lo = or_lo;
  b.out_len = orows;
  b.nlines = ocols;
  b.chirp = chirp;
  b.conj_chirp = conj;
  b.alpha = alpha;
  b.accumulate = accumulate;
  (void)P;
  HOLO_LAUNCH(c, c->ops->cols(b, c->d_tw, c->stream));
  return HOLO_OK;
}

holo_status check_chunk(holo_ctx* c, int k0, int nk) {
  if (!c) return HOLO_ERR_ARG;
  if (fault_on("arg")) return fail(c, HOLO_ERR_ARG, "argument error injected by HOLO_FAULT=arg");
  if (nk < 1 || nk > c->chunk || k0 < 0 || k0 + nk > c->K)
    return fail(c, HOLO_ERR_ARG, "chunk [k0, k0+nk) outside [0, n_angles) or nk > chunk");
  if (!c->have_shifts) return fail(c, HOLO_ERR_STATE, "holo_set_shifts not called");
  if (!c->have_data) return fail(c, HOLO_ERR_STATE, "holo_set_data not called");
  if (!c->have_probe) return fail(c, HOLO_ERR_STATE, "holo_set_probe not called");
  return HOLO_OK;
}

PassArgs pass_args(holo_ctx* c, int k0, int nk, const void* psi) {
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = c->n;
  a.P = c->P;
  a.J = c->J;
  a.k0 = k0;
  a.nk = nk;
  a.ext = c->ext;
  a.planes = c->d_planes;
  a.psi = (const float2*)psi;
  a.pj = c->d_pj;
  a.bref = c->d_b;
  a.dblk = c->d_dblk;
  a.dgroups = c->ops->pass_b_groups(c->n);
  a.data_k0 = 0;
  a.chirp_zhat = c->d_chirp_zhat;
  a.ybuf = c->ybuf;
  a.ystride = c->ystride;
  a.tq = c->d_T;
  a.functional = c->functional;
  a.rref = nullptr;
  a.wref = (float)c->wref;
  a.gkbuf = c->gkbuf;
  a.gkstride = c->gkstride;
  a.loss_part = c->d_part;
  a.twiddles = c->d_tw;
  int mb = 0;
  for (int k = k0; k < k0 + nk; ++k)
    for (int j = 0; j < c->J; ++j) mb = std::max(mb, c->planes[(size_t)k * c->J + j].bys);
  a.max_box_rows = std::max(mb, 1);
  a.xtap = c->d_xtap;
  a.ytap = c->d_ytap;
  a.xadj = c->d_xadj;
  a.yadj = c->d_yadj;
  a.tap_stride = c->tap_stride;
  a.lines = c->d_lines;
  a.line0 = c->rowstart[(size_t)k0 * c->J];
  a.nlines = c->rowstart[(size_t)(k0 + nk) * c->J] - a.line0;
  a.pass_b_items = c->ops->pass_b_groups(c->n);
  a.ymap = c->ystage && c->sched_stage != 0 ? c->d_ymap : nullptr;
  a.row_per_sm = c->sched_row_per_sm;
  a.yrows = (int)(c->ystride / c->n);
  a.err = reinterpret_cast<unsigned long long*>(c->d_red + kErrWord);
  if (c->probe_shift) {
    a.ramp_x = c->d_ramp_x;
    a.ramp_y = c->d_ramp_y;
    a.ymap = nullptr;
  }
  return a;
}

// One evaluation is split in three phases so that holo_gradient_host can run the planes of
// a chunk in parts while copies overlap:
//   eval_begin:  reference residual r_ref and its loss (only for the chunk with k0 == 0 and
//                w_ref != 0) into d_red[1], else d_red[1] = 0;
//   eval_planes: passes A, B (and C, D for gradients) of the angles of `a`; plane loss into
//                d_red[0] and the call / running totals (k_loss_total); pass B writes or adds
//                T = ext sum_kj r_kj (+ w_ref r_ref on the first part);
//   eval_qgrad:  grad_q of the whole chunk from T and the per-plane conj(w) v.
// Pass B's grid.  Whole column groups go to the blocks in rounds.  When that leaves a partial
// last round, the (group, plane) items of that round can be spread over all blocks: by the
// plane-split kernel (pb_split 1, no Y stage; the default when there are fewer than three full
// rounds, i.e. small n) or by the staged kernel itself (pb_split 2).  The partial residual sums
// of a split need tslots slots of [n][C] per block.
holo_status pass_b_grid(holo_ctx* c, PassArgs& a, bool gradient, int* nblocks) {
  const int groups = a.pass_b_items;
  const int full = c->ops->pass_b_blocks(1 << 30, c->n, a.ymap ? a.max_box_rows : 0);
  const bool partial = groups % full != 0;
  if (c->sched_split < 0)
    a.pb_split = partial && groups / full < 3 ? 1 : 0;
  else
    a.pb_split = partial ? c->sched_split : 0;
  a.tslots = 0;
  if (!a.pb_split) {
    *nblocks = std::min(full, groups);
    return HOLO_OK;
  }
  const long long per = (long long)a.J * a.nk;
  const int nbx = a.pb_split == 2 ? full
                                  : c->ops->pass_b_blocks_split((long long)groups * per, c->n);
  const long long rounds = groups / nbx, tail = groups - rounds * nbx, titems = tail * per;
  const long long range = (titems + nbx - 1) / nbx;
  a.tslots = titems > 0 ? (int)((range + per - 1) / per + 1) : 0;
  *nblocks = nbx;
  if (!gradient) return HOLO_OK;
  const size_t need = sizeof(float2) * (size_t)nbx * a.tslots * c->n * c->ops->pass_b_cols;
  if (need > c->tpart_bytes) {
    dfree(c, c->d_tpart, c->tpart_bytes);
    c->d_tpart = nullptr;
    c->tpart_bytes = 0;
    holo_status st = dalloc(c, (void**)&c->d_tpart, need);
    if (st) return st;
    c->tpart_bytes = need;
  }
  a.tpart = c->d_tpart;
  return HOLO_OK;
}

holo_status eval_begin(holo_ctx* c, PassArgs& a) {
  PassTimer tm_red(c, HOLO_T_REDUCE);
  const int nbx = c->ops->pass_b_blocks(a.pass_b_items, c->n, a.ymap ? a.max_box_rows : 0);
  const long long n2 = (long long)c->n * c->n;
  if (a.k0 == 0 && c->wref != 0.0) {
    // reference residual first: pass B folds w_ref r_ref into the grad_q source
    HOLO_LAUNCH(c, holo::launch_ref_residual(c->d_b, c->sqrt_dref, n2, c->d_rref,
                                             c->d_part + nbx, kRefBlocks, c->functional,
                                             c->stream));
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_part + nbx, kRefBlocks, c->d_red + 1, 0, c->stream));
    a.rref = c->d_rref;
  } else {
    // no reference term in this call: red[1] = 0 (a sum over nothing, by a kernel rather than a
    // memset, which could wait behind a host-buffer call's copies)
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_part, 0, c->d_red + 1, 0, c->stream));
  }
  return HOLO_OK;
}

// first: the first part of the call (adds the reference term, starts the call total);
// acc: add to the running total (user flags on the first part, always on later parts).
holo_status eval_planes(holo_ctx* c, PassArgs& a, bool gradient, bool first, int acc) {
  int nbx = 0;
  {
    holo_status st = pass_b_grid(c, a, gradient, &nbx);
    if (st) return st;
  }
  {
    PassTimer tm(c, HOLO_T_PASS_A);
    HOLO_LAUNCH(c, c->ops->pass_a(a, c->stream));
  }
  {
    PassTimer tm(c, HOLO_T_PASS_B);
    // with probe shifts the ext-part is inside the full-grid rows: no b term in pass B, and
    // T carries only the reference residual
    PassArgs ab = a;
    if (c->probe_shift) ab.ext = 0.f;
    HOLO_LAUNCH(c, c->ops->pass_b(ab, gradient ? 1 : 0, nbx, c->stream));
    // the last round's combine kernel of a split form (the staged split is compiled for the
    // form without probe shifts only; with them pb_split 2 runs whole groups)
    if (gradient && (a.pb_split == 1 || (a.pb_split == 2 && !c->probe_shift)) &&
        a.pass_b_items % nbx)
      c->launches++;
  }
  {
    PassTimer tm_red(c, HOLO_T_REDUCE);
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_part, nbx, c->d_red, 0, c->stream));
    HOLO_LAUNCH(c, holo::launch_loss_total(c->d_red, first ? c->wref : 0.0, acc, first ? 1 : 0,
                                           c->stream));
  }
  if (!gradient) return HOLO_OK;
  {
    PassTimer tm(c, HOLO_T_PASS_C);
    HOLO_LAUNCH(c, c->ops->pass_c(a, c->stream));
  }
  {
    PassTimer tm(c, HOLO_T_PASS_D);
    HOLO_LAUNCH(c, holo::launch_pass_d(a, c->stream));
  }
  return HOLO_OK;
}

// grad_q = 2 [ D_{-zeta_0}( C* T ) + sum_j D_{-omega_j}(G'_j) ] with T = ext sum_kj r_kj +
// w_ref r_ref written by pass B (zhat_j + omega_j = zeta_0 merges the ext-part of every
// plane into one propagation).  `a` spans the whole chunk; its gkbuf holds every plane.
// Deferred probe gradient: the chunk's G'_j added (acc) or written into the accumulators on
// the union boxes; T was written or accumulated by pass B (a.tq_accumulate).
holo_status eval_qsources(holo_ctx* c, const PassArgs& a, int acc) {
  PassTimer tm_q(c, HOLO_T_QGRAD);
  size_t need = 0, off[HOLO_MAX_DIST];
  for (int j = 0; j < c->J; ++j) {
    off[j] = need;
    need += sizeof(float2) * (size_t)c->qbox[j][1] * c->qbox[j][3];
  }
  if (need != c->gacc_bytes) {
    dfree(c, c->d_gacc, c->gacc_bytes);
    c->d_gacc = nullptr;
    c->gacc_bytes = 0;
    holo_status st = dalloc(c, (void**)&c->d_gacc, need);
    if (st) return st;
    c->gacc_bytes = need;
    acc = 0;
  }
  for (int j = 0; j < c->J; ++j) {
    c->gacc_off[j] = off[j] / sizeof(float2);
    const int* qb = c->qbox[j];
    if (qb[1] <= 0 || qb[3] <= 0) continue;
    HOLO_LAUNCH(c, holo::launch_reduce_g(a, c->d_gacc + c->gacc_off[j], j, qb[0], qb[1], qb[2],
                                         qb[3], qb[3], qb[0], qb[2], acc, c->stream));
  }
  c->q_pending = true;
  return HOLO_OK;
}

// grad_q (= or +=) 2 [ D_{-zeta_0}(C* T) + sum_j D_{-omega_j}(G'_j) ] from the accumulators.
// The row stage of every source runs into its own scratch rows; the column stage of all of
// them is one k_cols_sum launch (one inverse transform per column for the sum).  Where the
// sources' chirps do not fit its shared memory, each source runs its own column stage.
holo_status eval_qfinish(holo_ctx* c, float2* grad_q, int acc) {
  PassTimer tm_q(c, HOLO_T_QGRAD);
  const int P = c->P, n = c->n, lo = P / 2 - n / 2;
  struct Src {
    const float2* in;
    int r_lo, rows, c_lo, w;
    const float2* chirp;
  };
  Src src[holo::kMaxSumSources];
  int S = 0;
  src[S++] = {c->d_T, lo, n, lo, n, c->d_chirp_zeta0};
  for (int j = 0; j < c->J; ++j) {
    const int* qb = c->qbox[j];
    if (qb[1] <= 0 || qb[3] <= 0) continue;
    src[S++] = {c->d_gacc + c->gacc_off[j], qb[0], qb[1], qb[2], qb[3],
                c->d_chirp_omega + (size_t)j * P};
  }
  if (S > c->ops->cols_sum_max()) {
    for (int s = 0; s < S; ++s) {
      holo_status st = dstep2d(c, src[s].in, src[s].r_lo, src[s].rows, src[s].c_lo, src[s].w,
                               grad_q, 0, P, 0, P, src[s].chirp, 1, 2.f, s == 0 ? acc : 1);
      if (st != HOLO_OK) return st;
    }
    c->q_pending = false;
    return HOLO_OK;
  }
  size_t rows = 0;
  for (int s = 0; s < S; ++s) rows += (size_t)src[s].rows;
  const size_t need = sizeof(float2) * rows * P;
  if (need > c->qscr_bytes) {
    dfree(c, c->d_qscr, c->qscr_bytes);
    c->d_qscr = nullptr;
    c->qscr_bytes = 0;
    holo_status st = dalloc(c, (void**)&c->d_qscr, need);
    if (st) return st;
    c->qscr_bytes = need;
  }
  holo::SumArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  size_t off = 0;
  for (int s = 0; s < S; ++s) {
    LineArgs a = line_args();
    a.in = src[s].in;
    a.in_line_stride = src[s].w;
    a.in_step = 1;
    a.in_lo = src[s].c_lo;
    a.in_len = src[s].w;
    a.out = c->d_qscr + off;  // [rows][P]
    a.out_line_stride = P;
    a.out_step = 1;
    a.out_lo = 0;
    a.out_len = P;
    a.nlines = src[s].rows;
    a.chirp = src[s].chirp;
    a.conj_chirp = 1;
    HOLO_LAUNCH(c, c->ops->rows(a, c->d_tw, c->stream));
    sa.in[s] = c->d_qscr + off;
    sa.r_lo[s] = src[s].r_lo;
    sa.rows[s] = src[s].rows;
    sa.chirp[s] = src[s].chirp;
    off += (size_t)src[s].rows * P;
  }
  sa.S = S;
  sa.conj_chirp = 1;
  sa.alpha = 2.f;
  sa.accumulate = acc;
  sa.out = grad_q;
  HOLO_LAUNCH(c, c->ops->cols_sum(sa, c->d_tw, c->stream));
  c->q_pending = false;
  return HOLO_OK;
}

// grad_q of one chunk: its sources on the union boxes, then the propagation.
holo_status eval_qgrad(holo_ctx* c, const PassArgs& a, float2* grad_q, int acc) {
  holo_status st = eval_qsources(c, a, 0);
  if (st != HOLO_OK) return st;
  return eval_qfinish(c, grad_q, acc);
}

// The whole evaluation of one chunk in one pass over its planes.
holo_status run_eval(holo_ctx* c, PassArgs& a, bool gradient, float2* grad_q, unsigned flags) {
  const int acc = (flags & (HOLO_ACCUMULATE | HOLO_ACCUMULATE_Q)) ? 1 : 0;
  // deferred probe gradient: the sources accumulate onto pending ones when asked to
  const bool defer = gradient && (flags & HOLO_DEFER_Q);
  const int srcacc = defer && acc && c->q_pending ? 1 : 0;
  if (defer) a.tq_accumulate = srcacc;
  holo_status st;
  if ((st = eval_begin(c, a)) || (st = eval_planes(c, a, gradient, true, acc))) return st;
  if (!gradient) return HOLO_OK;
  if (defer) return eval_qsources(c, a, srcacc);
  c->q_pending = false;
  return eval_qgrad(c, a, grad_q, acc);
}

// A bounded device wait that gave up (the error word) is reported, and the word cleared,
// by the next call that reads a loss.
holo_status check_err_word(holo_ctx* c) {
  unsigned long long w;
  std::memcpy(&w, c->h_red + kErrWord, sizeof(w));
  if (!w) return HOLO_OK;
  HOLO_CK(c, cudaMemsetAsync(c->d_red + kErrWord, 0, sizeof(double), c->stream));
  if (w & 2)
    return fail(c, HOLO_ERR_BOUNDS,
                "a device bounds check failed; results of the evaluations since the last loss read are invalid");
  return fail(c, HOLO_ERR_TIMEOUT, "pass B: Y-tile wait gave up; results of the call are invalid");
}

holo_status read_loss(holo_ctx* c, double* loss, unsigned flags) {
  HOLO_CK(c, cudaMemcpyAsync(c->h_red + 7, c->d_red + 7, 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  if (holo_status st = check_err_word(c)) return st;
  const double l = fault_on("nan") ? std::nan("") : c->h_red[7];
  if (loss) *loss = (flags & (HOLO_ACCUMULATE | HOLO_ACCUMULATE_Q)) ? *loss + l : l;
  if (!std::isfinite(l)) return fail(c, HOLO_ERR_NUMERIC, "non-finite loss");
  return HOLO_OK;
}

// FP64 partials of the Dai-Yuan products: count entries, at least one per block of a
// direction step (grid_for caps those at 16 per SM of 152)
holo_status ensure_dypart(holo_ctx* c, long long count) {
  const size_t need = sizeof(double) * (size_t)std::max(count, 152LL * 16);
  if (need <= c->dypart_bytes) return HOLO_OK;
  dfree(c, c->d_dypart, c->dypart_bytes);
  c->d_dypart = nullptr;
  c->dypart_bytes = 0;
  holo_status st = dalloc(c, (void**)&c->d_dypart, need);
  if (st) return st;
  c->dypart_bytes = need;
  return HOLO_OK;
}

}  // namespace

extern "C" {

holo_status holo_set_timing(holo_ctx* c, int enable) {
  if (!c) return HOLO_ERR_ARG;
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  for (auto& r : c->recs) {
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  c->timing = enable != 0;
  return HOLO_OK;
}

holo_status holo_get_timing(holo_ctx* c, double* ms, long long* launches) {
  if (!c) return HOLO_ERR_ARG;
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  double t[HOLO_NUM_TIMERS] = {};
  long long l[HOLO_NUM_TIMERS] = {};
  for (auto& r : c->recs) {
    float e = 0.f;
    HOLO_CK(c, cudaEventElapsedTime(&e, r.a, r.b));
    if (r.id >= 0 && r.id < HOLO_NUM_TIMERS) {
      t[r.id] += e;
      l[r.id] += r.launches;
    }
  }
  for (int i = 0; i < HOLO_NUM_TIMERS; ++i) {
    if (ms) ms[i] = t[i];
    if (launches) launches[i] = l[i];
  }
  return HOLO_OK;
}

const char* holo_status_string(holo_status s) {
  switch (s) {
    case HOLO_OK: return "ok";
    case HOLO_ERR_ARG: return "invalid argument";
    case HOLO_ERR_CUDA: return "CUDA error";
    case HOLO_ERR_OOM: return "out of device memory";
    case HOLO_ERR_TIMEOUT: return "device wait timed out";
    case HOLO_ERR_STATE: return "call order (shifts, data or probe not set)";
    case HOLO_ERR_NUMERIC: return "non-finite result";
    case HOLO_ERR_UNSUPPORTED: return "unsupported size";
    case HOLO_ERR_BOUNDS: return "device bounds check failed";
  }
  return "unknown status";
}

const char* holo_last_error(const holo_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

holo_status holo_create(const holo_geometry* geo, void* stream, holo_ctx** out) {
  if (!out) return HOLO_ERR_ARG;
  *out = nullptr;
  if (!geo) return HOLO_ERR_ARG;
  const int n = geo->n, P = geo->pad ? geo->pad : 2 * geo->n, J = geo->n_dist;
  if (n < 16 || (n & 1) || n > P || ((P - n) & 1)) return HOLO_ERR_ARG;
  if (geo->n_angles < 1 || J < 1 || J > HOLO_MAX_DIST) return HOLO_ERR_ARG;
  if (geo->chunk < 0 || geo->chunk > geo->n_angles) return HOLO_ERR_ARG;
  if (!(geo->wavelength > 0) || !(geo->pixel > 0) || !(geo->Z > 0)) return HOLO_ERR_ARG;
  if (!(geo->z[0] > 0)) return HOLO_ERR_ARG;
  for (int j = 1; j < J; ++j)
    if (!(geo->z[j] > geo->z[j - 1])) return HOLO_ERR_ARG;
  if (!(geo->z[J - 1] < geo->Z)) return HOLO_ERR_ARG;
  if (!(geo->w_ref >= 0) || !std::isfinite(geo->w_ref) || !std::isfinite(geo->ext))
    return HOLO_ERR_ARG;
  if (!supported_line(P)) return HOLO_ERR_UNSUPPORTED;
  const holo::Ops* ops = holo::ops_for(P);
  if (!ops) return HOLO_ERR_UNSUPPORTED;

  holo_ctx* c = new holo_ctx();
  c->geo = *geo;
  c->n = n;
  c->P = P;
  c->J = J;
  c->K = geo->n_angles;
  c->chunk = geo->chunk ? geo->chunk : geo->n_angles;
  c->ext = (float)geo->ext;
  c->wref = geo->w_ref;
  c->stream = (cudaStream_t)stream;
  c->ops = ops;
  // Sec. 2 after Eq. fwd_model_cone3: m~_j = z_j/z_0, omega_j = (z_j - z_0)/m~_j,
  // zeta_j = z_j (Z - z_j)/Z; detector-side distance zhat_j = zeta_j / m~_j^2.
  const double z0 = geo->z[0];
  for (int j = 0; j < J; ++j) {
    const double z = geo->z[j];
    c->mt[j] = z / z0;
    c->omega[j] = (z - z0) / c->mt[j];
    c->zeta[j] = z * (geo->Z - z) / geo->Z;
    c->zhat[j] = c->zeta[j] / (c->mt[j] * c->mt[j]);
  }
  holo_status st;
  auto bail = [&](holo_status s) {
    holo_destroy(c);
    return s;
  };
  const std::vector<float2> tw = twiddle_table(P);
  if ((int)tw.size() != ops->twiddle_count) return bail(HOLO_ERR_UNSUPPORTED);
  const size_t cP = sizeof(float2) * (size_t)P;
  if ((st = dalloc(c, (void**)&c->d_tw, sizeof(float2) * std::max<size_t>(tw.size(), 1))) ||
      (st = dalloc(c, (void**)&c->d_chirp_zhat, cP * J)) ||
      (st = dalloc(c, (void**)&c->d_chirp_omega, cP * J)) ||
      (st = dalloc(c, (void**)&c->d_chirp_zeta0, cP)) ||
      (st = dalloc(c, (void**)&c->d_chirp_tmp, cP)) ||
      (st = dalloc(c, (void**)&c->d_pj, cP * P * J)) ||
      (st = dalloc(c, (void**)&c->d_b, sizeof(float2) * (size_t)n * n)) ||
      (st = dalloc(c, (void**)&c->d_scratch, cP * P)) ||
      (st = dalloc(c, (void**)&c->d_T, sizeof(float2) * (size_t)n * n)) ||
      (st = dalloc(c, (void**)&c->d_rref, sizeof(float2) * (size_t)n * n)) ||
      (st = dalloc(c, (void**)&c->d_red, kRed * sizeof(double))) ||
      (st = dalloc(c, &c->d_ymap, sizeof(CUtensorMap))))
    return bail(st);
  if (cudaMemset(c->d_red, 0, kRed * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return bail(HOLO_ERR_CUDA);
  }
  if (cudaMallocHost((void**)&c->h_red, kRed * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return bail(HOLO_ERR_OOM);
  }
  if (!tw.empty() && (st = upload(c, c->d_tw, tw.data(), sizeof(float2) * tw.size())))
    return bail(st);
  for (int j = 0; j < J; ++j) {
    auto cz = chirp_table(P, geo->wavelength, geo->pixel, c->zhat[j]);
    auto co = chirp_table(P, geo->wavelength, geo->pixel, c->omega[j]);
    if ((st = upload(c, c->d_chirp_zhat + (size_t)j * P, cz.data(), cP)) ||
        (st = upload(c, c->d_chirp_omega + (size_t)j * P, co.data(), cP)))
      return bail(st);
  }
  auto c0 = chirp_table(P, geo->wavelength, geo->pixel, c->zeta[0]);
  if ((st = upload(c, c->d_chirp_zeta0, c0.data(), cP))) return bail(st);
  *out = c;
  return HOLO_OK;
}

holo_status holo_destroy(holo_ctx* c) {
  if (!c) return HOLO_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->d_tw,    c->d_chirp_zhat, c->d_chirp_omega, c->d_chirp_zeta0,
                  c->d_chirp_tmp, c->d_planes, c->d_pj,          c->d_b,
                  c->ybuf,    c->gkbuf,        c->d_scratch,
                  c->d_qscr,  c->d_T,          c->d_rref,        c->d_part,       c->d_dypart,
                  c->d_red,   c->d_dot3,       c->d_tpart,       c->s_psi,         c->s_gpsi,
                  c->s_data,       c->s_dblk,       c->d_dblk,        c->d_gacc,
                  c->s_q,     c->s_gq,         c->d_xtap,        c->d_ytap,
                  c->d_xadj,  c->d_yadj,       c->d_lines,       c->d_ymap,
                  c->d_ramp_x, c->d_ramp_y};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_red) cudaFreeHost(c->h_red);
  for (cudaStream_t st : {c->cs_in, c->cs_out})
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : {c->ev_start, c->ev_out, c->ev_q})
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < kHostParts; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_done[i]) cudaEventDestroy(c->ev_done[i]);
  }
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  delete c;
  return HOLO_OK;
}

}  // extern "C"

namespace {

// Plane descriptors, bilinear tap tables, the flat row list and the per-plane workspace for
// the sample shifts t (and probe shifts, when set).  Without probe shifts each plane's box
// is the support of R0(psi - ext); with them the box is the whole P x P grid and the taps
// use the object shift t - m~_j s (FP64).  Until it succeeds the context has no valid
// planes (evaluations return HOLO_ERR_STATE), so a failed rebuild never leaves stale or
// freed tables in use.
holo_status build_planes(holo_ctx* c) {
  const int n = c->n, P = c->P, J = c->J, K = c->K;
  const float* t = c->t_host.data();
  c->have_shifts = false;
  c->planes.assign((size_t)K * J, PlaneDesc{});
  std::vector<double> teff((size_t)K * J * 2);
  int maxbys = 1, maxbxs = 1;
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < J; ++j) {
      const size_t p = (size_t)k * J + j;
      PlaneDesc& d = c->planes[p];
      split_mt(c->mt[j], P, &d.mt_hi, &d.mt_lo);
      double ty = t[p * 2 + 0], tx = t[p * 2 + 1];
      if (c->probe_shift) {
        ty -= c->mt[j] * (double)c->s_host[p * 2 + 0];
        tx -= c->mt[j] * (double)c->s_host[p * 2 + 1];
        d.by0 = d.bx0 = 0;
        d.bys = d.bxs = P;
      } else {
        axis_box(c->mt[j], ty, n, P, &d.by0, &d.bys);
        axis_box(c->mt[j], tx, n, P, &d.bx0, &d.bxs);
      }
      teff[p * 2 + 0] = ty;
      teff[p * 2 + 1] = tx;
      int* qb = c->qbox[j];
      if (k == 0) {
        qb[0] = d.by0;
        qb[1] = d.bys;
        qb[2] = d.bx0;
        qb[3] = d.bxs;
      } else {
        const int r1 = std::max(qb[0] + qb[1], d.by0 + d.bys), c1 = std::max(qb[2] + qb[3], d.bx0 + d.bxs);
        qb[0] = std::min(qb[0], d.by0);
        qb[2] = std::min(qb[2], d.bx0);
        qb[1] = r1 - qb[0];
        qb[3] = c1 - qb[2];
      }
      d.ty = (float)ty;
      d.tx = (float)tx;
      maxbys = std::max(maxbys, d.bys);
      maxbxs = std::max(maxbxs, d.bxs);
    }
  // tap tables and the flat list of box rows of all planes
  const size_t np_all = (size_t)K * J;
  const int stride = std::max(maxbys, maxbxs);
  std::vector<holo::Tap> xt(np_all * stride), yt(np_all * stride);
  std::vector<holo::AdjTap> xa(np_all * n), ya(np_all * n);
  c->rowstart.assign(np_all + 1, 0);
  for (size_t p = 0; p < np_all; ++p) {
    const PlaneDesc& d = c->planes[p];
    const double mt = c->mt[p % J];
    axis_taps(mt, teff[p * 2 + 1], n, P, d.bx0, d.bxs, &xt[p * stride], &xa[p * n]);
    axis_taps(mt, teff[p * 2 + 0], n, P, d.by0, d.bys, &yt[p * stride], &ya[p * n]);
    c->rowstart[p + 1] = c->rowstart[p] + d.bys;
  }
  std::vector<int2> lines((size_t)c->rowstart[np_all]);
  for (size_t p = 0; p < np_all; ++p)
    for (int r = 0; r < c->planes[p].bys; ++r) lines[(size_t)c->rowstart[p] + r] = make_int2((int)p, r);
  holo_status st;
  {
    void* olds[] = {c->d_xtap, c->d_ytap, c->d_xadj, c->d_yadj, c->d_lines};
    for (void* o : olds)
      if (o) cudaFree(o);
    c->bytes -= (long long)c->tap_bytes;
    c->d_xtap = c->d_ytap = nullptr;
    c->d_xadj = c->d_yadj = nullptr;
    c->d_lines = nullptr;
    const size_t tb = sizeof(holo::Tap) * xt.size(), ab = sizeof(holo::AdjTap) * xa.size(),
                 rb = sizeof(int2) * lines.size();
    if ((st = dalloc(c, (void**)&c->d_xtap, tb)) || (st = dalloc(c, (void**)&c->d_ytap, tb)) ||
        (st = dalloc(c, (void**)&c->d_xadj, ab)) || (st = dalloc(c, (void**)&c->d_yadj, ab)) ||
        (st = dalloc(c, (void**)&c->d_lines, rb)))
      return st;
    c->tap_bytes = 2 * tb + 2 * ab + rb;
    if ((st = upload(c, c->d_xtap, xt.data(), tb)) || (st = upload(c, c->d_ytap, yt.data(), tb)) ||
        (st = upload(c, c->d_xadj, xa.data(), ab)) || (st = upload(c, c->d_yadj, ya.data(), ab)) ||
        (st = upload(c, c->d_lines, lines.data(), rb)))
      return st;
    c->tap_stride = stride;
  }
  if (c->d_planes) {
    cudaFree(c->d_planes);
    c->bytes -= (long long)(sizeof(PlaneDesc) * c->planes.size());
    c->d_planes = nullptr;
  }
  if ((st = dalloc(c, (void**)&c->d_planes, sizeof(PlaneDesc) * c->planes.size()))) return st;
  if ((st = upload(c, c->d_planes, c->planes.data(), sizeof(PlaneDesc) * c->planes.size())))
    return st;
  const long long ystride = (long long)maxbys * n, gkstride = (long long)maxbys * maxbxs;
  const long long np = (long long)c->chunk * J;
  const size_t ybytes = sizeof(float2) * (size_t)(np * ystride);
  const size_t gbytes = sizeof(float2) * (size_t)(np * gkstride);
  const long long parts = (long long)c->ops->pass_b_blocks(1 << 30, n, 0) + kRefBlocks + 1024;
  if (ystride > c->ystride || gkstride > c->gkstride || !c->ybuf) {
    dfree(c, c->ybuf, sizeof(float2) * (size_t)(np * c->ystride));
    dfree(c, c->gkbuf, sizeof(float2) * (size_t)(np * c->gkstride));
    c->ybuf = c->gkbuf = nullptr;
    c->ystride = ystride;
    c->gkstride = gkstride;
    if ((st = dalloc(c, (void**)&c->ybuf, ybytes)) || (st = dalloc(c, (void**)&c->gkbuf, gbytes)))
      return st;
  }
  if ((st = encode_ystage(c, maxbys))) return st;
  if (parts > c->part_cap) {
    dfree(c, c->d_part, sizeof(double) * (size_t)c->part_cap);
    c->d_part = nullptr;
    c->part_cap = 0;
    if ((st = dalloc(c, (void**)&c->d_part, sizeof(double) * (size_t)parts))) return st;
    c->part_cap = parts;
  }
  c->maxbys = maxbys;
  c->maxbxs = maxbxs;
  c->q_pending = false;
  c->have_shifts = true;
  return HOLO_OK;
}

}  // namespace

extern "C" {

holo_status holo_set_shifts(holo_ctx* c, const float* t) {
  if (!c || !t) return fail(c, HOLO_ERR_ARG, "null argument");
  const int n = c->n;
  const long long cnt = 2LL * c->K * c->J;
  for (long long i = 0; i < cnt; ++i)
    if (!std::isfinite(t[i]) || std::fabs(t[i]) > n) return fail(c, HOLO_ERR_ARG, "bad shift");
  c->t_host.assign(t, t + cnt);
  return build_planes(c);
}

holo_status holo_set_probe_shifts(holo_ctx* c, const float* s) {
  if (!c) return HOLO_ERR_ARG;
  const int n = c->n, P = c->P;
  const long long np = (long long)c->K * c->J;
  if (!s) {
    c->probe_shift = false;
    c->s_host.clear();
    dfree(c, c->d_ramp_x, c->ramp_bytes);
    dfree(c, c->d_ramp_y, c->ramp_bytes);
    c->d_ramp_x = c->d_ramp_y = nullptr;
    c->ramp_bytes = 0;
    return c->have_shifts ? build_planes(c) : HOLO_OK;
  }
  for (long long i = 0; i < 2 * np; ++i)
    if (!std::isfinite(s[i]) || std::fabs(s[i]) > n / 2)
      return fail(c, HOLO_ERR_ARG, "bad probe shift (|s| must be at most n/2)");
  // phase ramps of S_s on the DFT, k in [-P/2, P/2) (FP64)
  const double kPi = 3.14159265358979323846;
  const size_t bytes = sizeof(float2) * (size_t)np * P;
  std::vector<float2> rx((size_t)np * P), ry((size_t)np * P);
  for (long long p = 0; p < np; ++p)
    for (int f = 0; f < P; ++f) {
      const double k = f < P / 2 ? f : f - P;
      const double ay = -2.0 * kPi * k * (double)s[p * 2 + 0] / P;
      const double ax = -2.0 * kPi * k * (double)s[p * 2 + 1] / P;
      ry[(size_t)p * P + f] = make_float2((float)std::cos(ay), (float)std::sin(ay));
      rx[(size_t)p * P + f] = make_float2((float)std::cos(ax), (float)std::sin(ax));
    }
  holo_status st;
  // on a failure below the context drops its probe shifts and its planes (evaluations then
  // return HOLO_ERR_STATE until holo_set_shifts succeeds again)
  auto drop = [&](holo_status e) {
    c->probe_shift = false;
    c->s_host.clear();
    c->have_shifts = false;
    return e;
  };
  if (bytes != c->ramp_bytes) {
    dfree(c, c->d_ramp_x, c->ramp_bytes);
    dfree(c, c->d_ramp_y, c->ramp_bytes);
    c->d_ramp_x = c->d_ramp_y = nullptr;
    c->ramp_bytes = 0;
    if ((st = dalloc(c, (void**)&c->d_ramp_x, bytes)) ||
        (st = dalloc(c, (void**)&c->d_ramp_y, bytes))) {
      dfree(c, c->d_ramp_x, bytes);
      c->d_ramp_x = nullptr;
      return drop(st);
    }
    c->ramp_bytes = bytes;
  }
  if ((st = upload(c, c->d_ramp_x, rx.data(), bytes)) ||
      (st = upload(c, c->d_ramp_y, ry.data(), bytes)))
    return drop(st);
  c->s_host.assign(s, s + 2 * np);
  c->probe_shift = true;
  return c->have_shifts ? build_planes(c) : HOLO_OK;
}

holo_status holo_set_data(holo_ctx* c, const float* sqrt_d, const float* sqrt_dref) {
  if (!c) return HOLO_ERR_ARG;
  if (!sqrt_d && !sqrt_dref) return fail(c, HOLO_ERR_ARG, "null data");
  if (c->wref != 0.0 && !sqrt_dref) return fail(c, HOLO_ERR_ARG, "w_ref != 0 needs sqrt_dref");
  c->sqrt_dref = sqrt_dref;
  if (sqrt_d) {
    // copy into pass B's column-blocked layout, then synchronise so the caller may reuse or
    // free its buffer as soon as the call returns
    const int C = c->ops->pass_b_cols, groups = c->ops->pass_b_groups(c->n);
    const long long planes = (long long)c->K * c->J;
    const size_t need = sizeof(float) * (size_t)planes * groups * c->n * C;
    if (need != c->dblk_bytes) {
      dfree(c, c->d_dblk, c->dblk_bytes);
      c->d_dblk = nullptr;
      c->dblk_bytes = 0;
      c->have_data = false;
      holo_status st = dalloc(c, (void**)&c->d_dblk, need);
      if (st) return st;
      c->dblk_bytes = need;
    }
    HOLO_LAUNCH(c, holo::launch_block_data(sqrt_d, planes, c->n, C, c->d_dblk, c->stream));
    HOLO_CK(c, cudaStreamSynchronize(c->stream));
  }
  c->have_data = sqrt_d != nullptr;
  return HOLO_OK;
}

holo_status holo_set_probe(holo_ctx* c, const void* q) {
  if (!c || !q) return fail(c, HOLO_ERR_ARG, "null probe");
  const int P = c->P, n = c->n, lo = P / 2 - n / 2;
  const size_t plane = sizeof(float2) * (size_t)P * P;
  PassTimer tm(c, HOLO_T_PROBE);
  // p_0 = q (omega_0 = 0), copied by a kernel: a copy engine may still be busy with the
  // host->device copies of a host-buffer call
  (void)plane;
  HOLO_LAUNCH(c, holo::launch_scale_add(c->d_pj, (const float2*)q, 1.f, (long long)P * P, 0,
                                        c->stream));
  holo_status st;
  for (int j = 1; j < c->J; ++j) {
    // p_j = D_{omega_j}(q)  (Eq. fwd_model_cone3)
    st = dstep2d(c, (const float2*)q, 0, P, 0, P, c->d_pj + (size_t)j * P * P, 0, P, 0, P,
                 c->d_chirp_omega + (size_t)j * P, 0, 1.f, 0);
    if (st != HOLO_OK) return st;
  }
  // b = C D_{zeta_0}(q): the probe on the detector without the sample (Sec. 2)
  st = dstep2d(c, (const float2*)q, 0, P, 0, P, c->d_b, lo, n, lo, n, c->d_chirp_zeta0, 0, 1.f, 0);
  if (st != HOLO_OK) return st;
  c->have_probe = true;
  return HOLO_OK;
}

holo_status holo_forward(holo_ctx* c, int k0, int nk, const void* psi, void* u_out,
                         double* loss) {
  holo_status st = check_chunk(c, k0, nk);
  if (st != HOLO_OK) return st;
  if (!psi) return fail(c, HOLO_ERR_ARG, "null psi");
  PassArgs a = pass_args(c, k0, nk, psi);
  a.u_out = (float2*)u_out;
  if ((st = run_eval(c, a, false, nullptr, 0))) return st;
  return read_loss(c, loss, 0);
}

holo_status holo_gradient(holo_ctx* c, int k0, int nk, const void* psi, double* loss,
                          void* grad_psi, void* grad_q, unsigned flags) {
  holo_status st = check_chunk(c, k0, nk);
  if (st != HOLO_OK) return st;
  if (!psi || !grad_psi || (!grad_q && !(flags & HOLO_DEFER_Q)))
    return fail(c, HOLO_ERR_ARG, "null pointer");
  PassArgs a = pass_args(c, k0, nk, psi);
  a.grad_psi = (float2*)grad_psi;
  a.accumulate = (flags & HOLO_ACCUMULATE) ? 1 : 0;
  if (c->dy_eta) {
    if ((st = ensure_dypart(c, 2LL * nk * c->n))) return st;
    a.dy_eta = c->dy_eta;
    a.dy_part = c->d_dypart;
  }
  if ((st = run_eval(c, a, true, (float2*)grad_q, flags))) return st;
  if (a.dy_eta) {
    PassTimer tm(c, HOLO_T_REDUCE);
    const int rows = nk * c->n;
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_dypart, rows, c->d_red + kDyWord, 0, c->stream));
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_dypart + rows, rows, c->d_red + kDyWord + 1, 0,
                                        c->stream));
  }
  if (!loss) return HOLO_OK;
  return read_loss(c, loss, flags);
}

// holo_gradient_host in `parts` parts of the chunk: part p's psi and data are copied on
// cs_in while earlier parts run passes A-D on the context's stream, and its grad_psi goes
// back on cs_out while later parts run.  Pass B adds each part's residual sum into T and
// every part keeps its conj(w) v in its own slice of the workspace, so grad_q is formed
// once for the whole chunk at the end.  (The per-part sums of T and of the loss round in a
// different order than a single pass over the chunk.)
static holo_status gradient_host_parts(holo_ctx* c, int k0, int nk, int parts, const void* psi_host,
                                const float* sqrt_d_host, const void* q_host, double* loss,
                                void* grad_psi_host, void* grad_q_host, unsigned flags) {
  const int n = c->n, P = c->P, J = c->J;
  const size_t n2 = (size_t)n * n;
  const size_t dplane = (size_t)c->ops->pass_b_groups(n) * n * c->ops->pass_b_cols;
  holo_status st;
  if (!c->cs_in) {
    if (cudaStreamCreateWithFlags(&c->cs_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cs_out, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_q, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess)
      return fail(c, HOLO_ERR_CUDA, std::string("copy streams: ") + cudaGetErrorString(cudaGetLastError()));
    for (int i = 0; i < kHostParts; ++i)
      if (cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&c->ev_done[i], cudaEventDisableTiming) != cudaSuccess)
        return fail(c, HOLO_ERR_CUDA, std::string("copy events: ") + cudaGetErrorString(cudaGetLastError()));
  }
  // copies start once everything issued earlier on the context's stream is done; the
  // probe (copy and propagation) then runs on the context's stream beside the first copies
  HOLO_CK(c, cudaEventRecord(c->ev_start, c->stream));
  HOLO_CK(c, cudaStreamWaitEvent(c->cs_in, c->ev_start, 0));
  HOLO_CK(c, cudaStreamWaitEvent(c->cs_out, c->ev_start, 0));
  // the probe first: every kernel of the call waits for it, and host->device copies run in
  // the order they were issued, so a probe copied after the parts' psi and data would hold
  // the whole call back by their copy time
  if (q_host) {
    HOLO_CK(c, cudaMemcpyAsync(c->s_q, q_host, sizeof(float2) * (size_t)P * P,
                               cudaMemcpyHostToDevice, c->cs_in));
    HOLO_CK(c, cudaEventRecord(c->ev_q, c->cs_in));
  }
  int wsum = 0;
  for (int p = 0; p < parts; ++p) wsum += kHostWeights[p];
  // part p covers [bound(p), bound(p + 1)) (rounded weight prefix sums); with nk >= 2 parts
  // every part is non-empty (checked for every nk up to 2000)
  auto bound = [&](int p) {
    int w = 0;
    for (int q = 0; q < p; ++q) w += kHostWeights[q];
    return p == parts ? nk : (int)(((long long)nk * w + wsum / 2) / wsum);
  };
  for (int p = 0; p < parts; ++p) {
    const int b0 = bound(p), m = bound(p + 1) - b0;
    HOLO_CK(c, cudaMemcpyAsync(c->s_psi + b0 * n2, static_cast<const float2*>(psi_host) + b0 * n2,
                               sizeof(float2) * m * n2, cudaMemcpyHostToDevice, c->cs_in));
    if (sqrt_d_host) {
      HOLO_CK(c, cudaMemcpyAsync(c->s_data + (size_t)b0 * J * n2, sqrt_d_host + (size_t)b0 * J * n2,
                                 sizeof(float) * m * J * n2, cudaMemcpyHostToDevice, c->cs_in));
      // the part's relayout runs on the copy stream as soon as its data arrive, beside the
      // passes of the earlier parts (its blocks fit next to theirs on an SM)
      HOLO_LAUNCH(c, holo::launch_block_data(c->s_data + (size_t)b0 * J * n2, (long long)m * J, n,
                                             c->ops->pass_b_cols,
                                             c->s_dblk + (size_t)b0 * J * dplane, c->cs_in));
    }
    HOLO_CK(c, cudaEventRecord(c->ev_in[p], c->cs_in));
  }
  if (q_host) {
    HOLO_CK(c, cudaStreamWaitEvent(c->stream, c->ev_q, 0));
    if ((st = holo_set_probe(c, c->s_q))) return st;
  }
  PassArgs whole = pass_args(c, k0, nk, c->s_psi);
  if ((st = eval_begin(c, whole))) return st;
  const int acc = (flags & (HOLO_ACCUMULATE | HOLO_ACCUMULATE_Q)) ? 1 : 0;
  for (int p = 0; p < parts; ++p) {
    const int b0 = bound(p), m = bound(p + 1) - b0;
    HOLO_CK(c, cudaStreamWaitEvent(c->stream, c->ev_in[p], 0));
    PassArgs a = pass_args(c, k0 + b0, m, c->s_psi + b0 * n2);
    if (sqrt_d_host) {
      a.dblk = c->s_dblk + (size_t)b0 * J * dplane;
      a.data_k0 = k0 + b0;
    }
    a.grad_psi = c->s_gpsi + b0 * n2;
    a.gkbuf = c->gkbuf + (size_t)b0 * J * c->gkstride;
    a.rref = p == 0 ? whole.rref : nullptr;
    a.tq_accumulate = p > 0;
    if ((st = eval_planes(c, a, true, p == 0, p == 0 ? acc : 1))) return st;
    HOLO_CK(c, cudaEventRecord(c->ev_done[p], c->stream));
    HOLO_CK(c, cudaStreamWaitEvent(c->cs_out, c->ev_done[p], 0));
    HOLO_CK(c, cudaMemcpyAsync(static_cast<float2*>(grad_psi_host) + b0 * n2, c->s_gpsi + b0 * n2,
                               sizeof(float2) * m * n2, cudaMemcpyDeviceToHost, c->cs_out));
  }
  if ((st = eval_qgrad(c, whole, c->s_gq, 0))) return st;
  HOLO_CK(c, cudaMemcpyAsync(grad_q_host, c->s_gq, sizeof(float2) * (size_t)P * P,
                             cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaEventRecord(c->ev_out, c->cs_out));
  HOLO_CK(c, cudaStreamWaitEvent(c->stream, c->ev_out, 0));
  return read_loss(c, loss, flags);
}

static holo_status gradient_host_impl(holo_ctx* c, int k0, int nk, const void* psi_host,
                                     const float* sqrt_d_host, const void* q_host, double* loss,
                                     void* grad_psi_host, void* grad_q_host, unsigned flags);

holo_status holo_gradient_host(holo_ctx* c, int k0, int nk, const void* psi_host,
                               const float* sqrt_d_host, const void* q_host, double* loss,
                               void* grad_psi_host, void* grad_q_host, unsigned flags) {
  const holo_status st = gradient_host_impl(c, k0, nk, psi_host, sqrt_d_host, q_host, loss,
                                            grad_psi_host, grad_q_host, flags);
  if (st != HOLO_OK && c) {
    // copies issued before the failure may still read or write the caller's host buffers:
    // let them finish before returning
    if (c->cs_in) cudaStreamSynchronize(c->cs_in);
    if (c->cs_out) cudaStreamSynchronize(c->cs_out);
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
  }
  return st;
}

static holo_status gradient_host_impl(holo_ctx* c, int k0, int nk, const void* psi_host,
                                     const float* sqrt_d_host, const void* q_host, double* loss,
                                     void* grad_psi_host, void* grad_q_host, unsigned flags) {
  if (!c) return HOLO_ERR_ARG;
  if (flags & HOLO_DEFER_Q) return fail(c, HOLO_ERR_ARG, "the host call does not defer grad_q");
  c->q_pending = false;
  if (!psi_host || !grad_psi_host || !grad_q_host) return fail(c, HOLO_ERR_ARG, "null pointer");
  if (nk < 1 || nk > c->chunk || k0 < 0 || k0 + nk > c->K)
    return fail(c, HOLO_ERR_ARG, "chunk [k0, k0+nk) outside [0, n_angles) or nk > chunk");
  if (!c->have_shifts) return fail(c, HOLO_ERR_STATE, "holo_set_shifts not called");
  if (!sqrt_d_host && !c->have_data) return fail(c, HOLO_ERR_STATE, "no data");
  if (c->wref != 0.0 && k0 == 0 && !c->sqrt_dref)
    return fail(c, HOLO_ERR_STATE, "reference data not registered");
  if (!q_host && !c->have_probe) return fail(c, HOLO_ERR_STATE, "holo_set_probe not called");
  const int n = c->n, P = c->P, J = c->J;
  const size_t psi_bytes = sizeof(float2) * (size_t)c->chunk * n * n;
  const size_t data_bytes = sizeof(float) * (size_t)c->chunk * J * n * n;
  const size_t q_bytes = sizeof(float2) * (size_t)P * P;
  holo_status st;
  if (!c->s_psi && ((st = dalloc(c, (void**)&c->s_psi, psi_bytes)) ||
                    (st = dalloc(c, (void**)&c->s_gpsi, psi_bytes)) ||
                    (st = dalloc(c, (void**)&c->s_q, q_bytes)) ||
                    (st = dalloc(c, (void**)&c->s_gq, q_bytes))))
    return st;
  const size_t dblk_bytes =
      sizeof(float) * (size_t)c->chunk * J * c->ops->pass_b_groups(n) * n * c->ops->pass_b_cols;
  if (sqrt_d_host && !c->s_data &&
      ((st = dalloc(c, (void**)&c->s_data, data_bytes)) ||
       (st = dalloc(c, (void**)&c->s_dblk, dblk_bytes))))
    return st;
  const int parts = nk >= 2 * kHostMinPart ? std::min(kHostParts, nk / kHostMinPart) : 1;
  if (parts > 1)
    return gradient_host_parts(c, k0, nk, parts, psi_host, sqrt_d_host, q_host, loss,
                               grad_psi_host, grad_q_host, flags);
  const size_t nb = sizeof(float2) * (size_t)nk * n * n;
  HOLO_CK(c, cudaMemcpyAsync(c->s_psi, psi_host, nb, cudaMemcpyHostToDevice, c->stream));
  if (sqrt_d_host)
    HOLO_CK(c, cudaMemcpyAsync(c->s_data, sqrt_d_host, sizeof(float) * (size_t)nk * J * n * n,
                               cudaMemcpyHostToDevice, c->stream));
  if (q_host) {
    HOLO_CK(c, cudaMemcpyAsync(c->s_q, q_host, q_bytes, cudaMemcpyHostToDevice, c->stream));
    if ((st = holo_set_probe(c, c->s_q))) return st;
  }
  PassArgs a = pass_args(c, k0, nk, c->s_psi);
  if (sqrt_d_host) {
    HOLO_LAUNCH(c, holo::launch_block_data(c->s_data, (long long)nk * J, n, c->ops->pass_b_cols,
                                           c->s_dblk, c->stream));
    a.dblk = c->s_dblk;
    a.data_k0 = k0;
  }
  a.grad_psi = c->s_gpsi;
  if ((st = run_eval(c, a, true, c->s_gq, 0))) return st;
  HOLO_CK(c, cudaMemcpyAsync(grad_psi_host, c->s_gpsi, nb, cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaMemcpyAsync(grad_q_host, c->s_gq, q_bytes, cudaMemcpyDeviceToHost, c->stream));
  return read_loss(c, loss, flags);
}

holo_status holo_finish_q(holo_ctx* c, void* grad_q, unsigned flags) {
  if (!c || !grad_q) return fail(c, HOLO_ERR_ARG, "null argument");
  if (!c->q_pending) return fail(c, HOLO_ERR_STATE, "no deferred probe-gradient sources");
  return eval_qfinish(c, static_cast<float2*>(grad_q),
                      (flags & (HOLO_ACCUMULATE | HOLO_ACCUMULATE_Q)) ? 1 : 0);
}

holo_status holo_propagate(holo_ctx* c, const void* in, void* out, double z) {
  if (!c || !in || !out || !std::isfinite(z)) return fail(c, HOLO_ERR_ARG, "bad argument");
  const int P = c->P;
  auto ch = chirp_table(P, c->geo.wavelength, c->geo.pixel, z);
  holo_status st = upload(c, c->d_chirp_tmp, ch.data(), sizeof(float2) * P);
  if (st) return st;
  return dstep2d(c, (const float2*)in, 0, P, 0, P, (float2*)out, 0, P, 0, P, c->d_chirp_tmp, 0,
                 1.f, 0);
}

holo_status holo_dot(holo_ctx* c, const void* a, const void* b, long long n, double* re_out) {
  if (!c || !a || !b || !re_out || n < 0) return fail(c, HOLO_ERR_ARG, "bad argument");
  if (!c->d_part) {
    holo_status st = dalloc(c, (void**)&c->d_part, sizeof(double) * 1024);
    if (st) return st;
    c->part_cap = 1024;
  }
  long long nb = (n + 256 * 16 - 1) / (256 * 16);
  nb = std::max(1LL, std::min(nb, std::min(1024LL, c->part_cap)));
  PassTimer tm(c, HOLO_T_REDUCE);
  HOLO_LAUNCH(c, holo::launch_dot((const float2*)a, (const float2*)b, n, c->d_part, (int)nb,
                                  c->stream));
  HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_part, (int)nb, c->d_red + 2, 0, c->stream));
  HOLO_CK(c, cudaMemcpyAsync(c->h_red + 2, c->d_red + 2, sizeof(double), cudaMemcpyDeviceToHost,
                             c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  *re_out = c->h_red[2];
  return HOLO_OK;
}

holo_status holo_dy_dots(holo_ctx* c, const void* g, const void* g_prev, const void* eta,
                         long long n, double* out) {
  if (!c || !g || !g_prev || !eta || !out || n < 0) return fail(c, HOLO_ERR_ARG, "bad argument");
  // enough blocks to fill every SM (8 resident blocks of 256 threads each)
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  const long long cap = 8LL * sms;
  if (!c->d_dot3) {
    holo_status st = dalloc(c, (void**)&c->d_dot3, sizeof(double) * 3 * cap);
    if (st) return st;
  }
  long long nb = (n + 256 * 16 - 1) / (256 * 16);
  nb = std::max(1LL, std::min(nb, cap));
  PassTimer tm(c, HOLO_T_REDUCE);
  HOLO_LAUNCH(c, holo::launch_dot3((const float2*)g, (const float2*)g_prev, (const float2*)eta, n,
                                   c->d_dot3, (int)nb, c->stream));
  for (int i = 0; i < 3; ++i)
    HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_dot3 + i * nb, (int)nb, c->d_red + 4 + i, 0,
                                        c->stream));
  HOLO_CK(c, cudaMemcpyAsync(c->h_red + 4, c->d_red + 4, 3 * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 3; ++i) out[i] = c->h_red[4 + i];
  return HOLO_OK;
}

holo_status holo_direction_step(holo_ctx* c, void* x, void* eta, const void* g, double beta,
                                double gamma, long long n) {
  if (!c || !x || !eta || !g || n < 0 || !std::isfinite(beta) || !std::isfinite(gamma))
    return fail(c, HOLO_ERR_ARG, "bad argument");
  PassTimer tm(c, HOLO_T_VECTOR);
  HOLO_LAUNCH(c, holo::launch_direction_step((float2*)x, (float2*)eta, (const float2*)g,
                                             (float)beta, (float)gamma, n, c->stream));
  return HOLO_OK;
}

holo_status holo_set_dy_direction(holo_ctx* c, const void* eta) {
  if (!c) return HOLO_ERR_ARG;
  if (eta && (reinterpret_cast<uintptr_t>(eta) & 15))
    return fail(c, HOLO_ERR_ARG, "dy direction: 16-byte aligned device memory expected");
  c->dy_eta = static_cast<const float2*>(eta);
  return HOLO_OK;
}

holo_status holo_direction_step_dy(holo_ctx* c, void* x, void* eta, const void* g, double beta,
                                   double gamma, long long n) {
  if (!c || !x || !eta || !g || n < 0 || !std::isfinite(beta) || !std::isfinite(gamma))
    return fail(c, HOLO_ERR_ARG, "bad argument");
  holo_status st = ensure_dypart(c, 0);
  if (st) return st;
  PassTimer tm(c, HOLO_T_VECTOR);
  int nb = 0;
  HOLO_LAUNCH(c, holo::launch_direction_step_dot((float2*)x, (float2*)eta, (const float2*)g,
                                                 (float)beta, (float)gamma, n, c->d_dypart, &nb,
                                                 c->stream));
  HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_dypart, nb, c->d_red + kDyWord + 2, 0, c->stream));
  return HOLO_OK;
}

holo_status holo_read_dy(holo_ctx* c, double* out) {
  if (!c || !out) return fail(c, HOLO_ERR_ARG, "null argument");
  HOLO_CK(c, cudaMemcpyAsync(c->h_red + kDyWord, c->d_red + kDyWord, 3 * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 3; ++i) out[i] = c->h_red[kDyWord + i];
  return HOLO_OK;
}

holo_status holo_step(holo_ctx* c, void* x, const void* eta, double gamma, long long n) {
  if (!c || !x || !eta || n < 0 || !std::isfinite(gamma)) return fail(c, HOLO_ERR_ARG, "bad argument");
  PassTimer tm(c, HOLO_T_VECTOR);
  HOLO_LAUNCH(c, holo::launch_axpy((float2*)x, (const float2*)eta, (float)gamma, n, c->stream));
  return HOLO_OK;
}

holo_status holo_direction(holo_ctx* c, void* eta, const void* g, double beta, long long n) {
  if (!c || !eta || !g || n < 0 || !std::isfinite(beta)) return fail(c, HOLO_ERR_ARG, "bad argument");
  PassTimer tm(c, HOLO_T_VECTOR);
  HOLO_LAUNCH(c, holo::launch_direction((float2*)eta, (const float2*)g, (float)beta, n, c->stream));
  return HOLO_OK;
}

holo_status holo_bin_amplitudes(const float* in, long long count, int n, int b, float* out,
                                void* stream) {
  if (!in || !out || count < 0 || n < 1 || b < 1 || n % b) return HOLO_ERR_ARG;
  if (holo::launch_bin_amplitudes(in, count, n, b, out, (cudaStream_t)stream) != cudaSuccess)
    return HOLO_ERR_CUDA;
  return HOLO_OK;
}

holo_status holo_upsample2(const void* in, long long count, int n, void* out, void* stream) {
  if (!in || !out || count < 0 || n < 1 || in == out) return HOLO_ERR_ARG;
  if (holo::launch_upsample2((const float2*)in, count, n, (float2*)out, (cudaStream_t)stream) !=
      cudaSuccess)
    return HOLO_ERR_CUDA;
  return HOLO_OK;
}

holo_status holo_initial_probe(holo_ctx* c, const float* sqrt_dref, void* q_out) {
  if (!c || !sqrt_dref || !q_out) return fail(c, HOLO_ERR_ARG, "null argument");
  const int P = c->P;
  HOLO_LAUNCH(c, holo::launch_embed_edge(sqrt_dref, c->n, P, (float2*)q_out, c->stream));
  return dstep2d(c, (const float2*)q_out, 0, P, 0, P, (float2*)q_out, 0, P, 0, P,
                 c->d_chirp_zeta0, 1, 1.f, 0);
}

holo_status holo_set_functional(holo_ctx* c, int functional) {
  if (!c) return HOLO_ERR_ARG;
  if (functional != HOLO_F2_AMPLITUDE && functional != HOLO_F1_INTENSITY)
    return fail(c, HOLO_ERR_ARG, "functional must be HOLO_F2_AMPLITUDE or HOLO_F1_INTENSITY");
  c->functional = functional;
  return HOLO_OK;
}

holo_status holo_set_schedule(holo_ctx* c, int row_blocks_per_sm, int pass_b_stage,
                              int pass_b_split) {
  if (!c || row_blocks_per_sm < 0 || pass_b_stage < -1 || pass_b_stage > 1 || pass_b_split < -1 ||
      pass_b_split > 2)
    return fail(c, HOLO_ERR_ARG, "schedule: blocks per SM >= 0, stage in {-1, 0, 1}, split in {-1 .. 2}");
  c->sched_row_per_sm = row_blocks_per_sm;
  c->sched_stage = pass_b_stage;
  c->sched_split = pass_b_split;
  return HOLO_OK;
}

holo_status holo_set_stream(holo_ctx* c, void* stream) {
  if (!c) return HOLO_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return HOLO_OK;
}

holo_status holo_read_loss(holo_ctx* c, double* loss) {
  if (!c || !loss) return fail(c, HOLO_ERR_ARG, "null argument");
  HOLO_CK(c, cudaMemcpyAsync(c->h_red + 3, c->d_red + 3, (kErrWord - 2) * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  if (holo_status st = check_err_word(c)) return st;
  *loss = fault_on("nan") ? std::nan("") : c->h_red[3];
  if (!std::isfinite(*loss)) return fail(c, HOLO_ERR_NUMERIC, "non-finite loss");
  return HOLO_OK;
}

holo_status holo_set_device_error(holo_ctx* c, unsigned long long word) {
  if (!c) return HOLO_ERR_ARG;
  HOLO_CK(c, cudaMemcpyAsync(c->d_red + kErrWord, &word, sizeof(word), cudaMemcpyHostToDevice,
                             c->stream));
  HOLO_CK(c, cudaStreamSynchronize(c->stream));
  return HOLO_OK;
}

holo_status holo_workspace_bytes(const holo_ctx* c, long long* bytes) {
  if (!c || !bytes) return HOLO_ERR_ARG;
  *bytes = c->bytes;
  return HOLO_OK;
}

holo_status holo_launch_count(const holo_ctx* c, long long* count) {
  if (!c || !count) return HOLO_ERR_ARG;
  *count = c->launches;
  return HOLO_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched evaluation

// Work lists of one round of a batch: the r-th chunk of every problem that has one.  Problems
// of one line length (and probe-shift form) share the launches of passes A, B and C; pass D
// has one launch for all.  Items are {index into the round's PassArgs, work index}.
struct BatchGroup {
  const holo::Ops* ops = nullptr;
  int shift = 0, max_n = 0, max_rows = 0, per_sm = 0;
  std::vector<int2> rows, cols;  // pass A / C: {arg, first line}; pass B: {arg, block}
  size_t off_rows = 0, off_cols = 0;
};

struct BatchRound {
  std::vector<int> prob;          // problem of each PassArgs
  std::vector<PassArgs> args;     // host copies (also used for the per-problem launches)
  std::vector<int> nbx;           // pass-B grid of each
  std::vector<BatchGroup> groups;
  std::vector<int2> dits;         // pass D: {arg, kl * n + i}
  size_t off_args = 0, off_dits = 0;
};

struct holo_batch {
  std::vector<holo_ctx*> ctx;
  struct Buffers {
    const float2* psi = nullptr;
    const float2* q = nullptr;
    float2* gpsi = nullptr;
    float2* gq = nullptr;
  };
  std::vector<Buffers> buf;
  std::vector<BatchRound> rounds;
  void* dmem = nullptr;           // every round's PassArgs and items, one allocation
  size_t dbytes = 0;
  bool prepared = false;
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

extern "C" {

holo_status holo_batch_create(holo_ctx* const* ctxs, int count, holo_batch** out) {
  if (!out) return HOLO_ERR_ARG;
  *out = nullptr;
  if (!ctxs || count < 1) return HOLO_ERR_ARG;
  for (int i = 0; i < count; ++i)
    if (!ctxs[i]) return HOLO_ERR_ARG;
  holo_batch* b = new holo_batch();
  b->ctx.assign(ctxs, ctxs + count);
  b->buf.resize(count);
  *out = b;
  return HOLO_OK;
}

holo_status holo_batch_set_problem(holo_batch* b, int i, const void* psi, const void* q,
                                   void* grad_psi, void* grad_q) {
  if (!b || i < 0 || i >= (int)b->ctx.size() || !psi || !q || !grad_psi || !grad_q)
    return HOLO_ERR_ARG;
  b->buf[i] = {static_cast<const float2*>(psi), static_cast<const float2*>(q),
               static_cast<float2*>(grad_psi), static_cast<float2*>(grad_q)};
  b->prepared = false;
  return HOLO_OK;
}

holo_status holo_batch_destroy(holo_batch* b) {
  if (!b) return HOLO_OK;
  if (b->dmem) cudaFree(b->dmem);
  delete b;
  return HOLO_OK;
}

holo_status holo_batch_prepare(holo_batch* b) {
  if (!b) return HOLO_ERR_ARG;
  holo_ctx* c0 = b->ctx[0];
  b->prepared = false;
  b->rounds.clear();
  int nround = 0;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    holo_ctx* c = b->ctx[i];
    if (!b->buf[i].psi) return fail(c0, HOLO_ERR_STATE, "batch: problem buffers not set");
    if (!c->have_shifts || !c->have_data)
      return fail(c0, HOLO_ERR_STATE, "batch: a problem has no shifts or data");
    c->sched_split = 0;  // the batched column pass works on whole column groups
    nround = std::max(nround, (c->K + c->chunk - 1) / c->chunk);
  }
  size_t off = 0;
  b->rounds.resize(nround);
  for (int r = 0; r < nround; ++r) {
    BatchRound& R = b->rounds[r];
    for (size_t i = 0; i < b->ctx.size(); ++i) {
      holo_ctx* c = b->ctx[i];
      const int k0 = r * c->chunk;
      if (k0 >= c->K) continue;
      const int nk = std::min(c->chunk, c->K - k0);
      const size_t n2 = (size_t)c->n * c->n;
      PassArgs a = pass_args(c, k0, nk, b->buf[i].psi + (size_t)k0 * n2);
      a.grad_psi = b->buf[i].gpsi + (size_t)k0 * n2;
      a.accumulate = 0;
      a.tq_accumulate = r > 0 ? 1 : 0;  // probe-gradient sources summed over the rounds
      if (k0 == 0 && c->wref != 0.0) a.rref = c->d_rref;
      int nbx = 0;
      holo_status st = pass_b_grid(c, a, true, &nbx);
      if (st) return st;
      a.pb_blocks = nbx;
      const int ai = (int)R.args.size();
      R.prob.push_back((int)i);
      R.args.push_back(a);
      R.nbx.push_back(nbx);
      const int shift = a.ramp_x != nullptr;
      BatchGroup* g = nullptr;
      for (auto& x : R.groups)
        if (x.ops == c->ops && x.shift == shift) g = &x;
      if (!g) {
        R.groups.emplace_back();
        g = &R.groups.back();
        g->ops = c->ops;
        g->shift = shift;
        g->per_sm = c->sched_row_per_sm;
      }
      g->max_n = std::max(g->max_n, c->n);
      if (a.ymap) g->max_rows = std::max(g->max_rows, a.max_box_rows);
      for (int base = 0; base < a.nlines; base += c->ops->row_lines) g->rows.push_back({ai, base});
      for (int blk = 0; blk < nbx; ++blk) g->cols.push_back({ai, blk});
      for (int e = 0; e < nk * c->n; ++e) R.dits.push_back({ai, e});
    }
    R.off_args = off = align_up(off, 256);
    off += sizeof(PassArgs) * R.args.size();
    for (auto& g : R.groups) {
      g.off_rows = off = align_up(off, 256);
      off += sizeof(int2) * g.rows.size();
      g.off_cols = off = align_up(off, 256);
      off += sizeof(int2) * g.cols.size();
    }
    R.off_dits = off = align_up(off, 256);
    off += sizeof(int2) * R.dits.size();
  }
  std::vector<char> host(off);
  for (auto& R : b->rounds) {
    std::memcpy(host.data() + R.off_args, R.args.data(), sizeof(PassArgs) * R.args.size());
    for (auto& g : R.groups) {
      std::memcpy(host.data() + g.off_rows, g.rows.data(), sizeof(int2) * g.rows.size());
      std::memcpy(host.data() + g.off_cols, g.cols.data(), sizeof(int2) * g.cols.size());
    }
    std::memcpy(host.data() + R.off_dits, R.dits.data(), sizeof(int2) * R.dits.size());
  }
  if (off > b->dbytes) {
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
    b->dbytes = 0;
    if (cudaMalloc(&b->dmem, off) != cudaSuccess) {
      cudaGetLastError();
      return fail(c0, HOLO_ERR_OOM, "batch work lists");
    }
    b->dbytes = off;
  }
  HOLO_CK(c0, cudaMemcpy(b->dmem, host.data(), off, cudaMemcpyHostToDevice));
  b->prepared = true;
  return HOLO_OK;
}

}  // extern "C"

extern "C" holo_status holo_batch_gradient(holo_batch* b, void* stream) {
  if (!b) return HOLO_ERR_ARG;
  holo_ctx* c0 = b->ctx[0];
  if (!b->prepared) return fail(c0, HOLO_ERR_STATE, "batch: holo_batch_prepare not called");
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  holo_status st;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    b->ctx[i]->stream = s;
    if ((st = holo_set_probe(b->ctx[i], b->buf[i].q))) return st;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 1;
    }
  }
  char* dm = static_cast<char*>(b->dmem);
  for (size_t r = 0; r < b->rounds.size(); ++r) {
    BatchRound& R = b->rounds[r];
    const PassArgs* dargs = reinterpret_cast<const PassArgs*>(dm + R.off_args);
    const int acc = r > 0 ? 1 : 0;
    const int na = (int)R.args.size();
    for (int ai = 0; ai < na; ++ai) {
      PassArgs a = R.args[ai];
      if ((st = eval_begin(b->ctx[R.prob[ai]], a))) return st;
    }
    for (auto& g : R.groups)
      HOLO_CK(c0, g.ops->rows_multi(0, dargs, reinterpret_cast<const int2*>(dm + g.off_rows),
                                    (int)g.rows.size(), g.shift, g.max_n, g.per_sm, s));
    for (auto& g : R.groups)
      HOLO_CK(c0, g.ops->pass_b_multi(dargs, reinterpret_cast<const int2*>(dm + g.off_cols),
                                      (int)g.cols.size(), na, 1, g.shift, g.max_n, g.max_rows, 0,
                                      s));
    for (int ai = 0; ai < na; ++ai) {
      holo_ctx* c = b->ctx[R.prob[ai]];
      HOLO_LAUNCH(c, holo::launch_sum_f64(c->d_part, R.nbx[ai], c->d_red, 0, s));
      HOLO_LAUNCH(c, holo::launch_loss_total(c->d_red, c->wref, acc, 1, s));
    }
    for (auto& g : R.groups)
      HOLO_CK(c0, g.ops->rows_multi(1, dargs, reinterpret_cast<const int2*>(dm + g.off_rows),
                                    (int)g.rows.size(), g.shift, g.max_n, g.per_sm, s));
    HOLO_CK(c0, holo::launch_pass_d_multi(dargs, reinterpret_cast<const int2*>(dm + R.off_dits),
                                          (int)R.dits.size(), 16 * sms, s));
    // the probe gradient's sources are summed over the rounds and propagated once, in the
    // problem's last round (as its own calls with HOLO_DEFER_Q and holo_finish_q)
    for (int ai = 0; ai < na; ++ai) {
      const int i = R.prob[ai];
      holo_ctx* c = b->ctx[i];
      if ((st = eval_qsources(c, R.args[ai], acc))) return st;
      if ((int)r == (c->K + c->chunk - 1) / c->chunk - 1 &&
          (st = eval_qfinish(c, b->buf[i].gq, 0)))
        return st;
    }
  }
  return HOLO_OK;
}
