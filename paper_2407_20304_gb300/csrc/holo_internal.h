// Internal declarations shared by the C-ABI layer and the per-line-length kernel units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "holo.h"

namespace holo {

// One (angle k, distance j) plane: resample parameters and the bounding box of the
// support of R0(psi - ext) on the P x P grid (rows [by0, by0+bys), cols [bx0, bx0+bxs)).
// m~ is split into a high part with few significant bits (so m_hi * integer is exact in
// FP32) and a low part; see axis_tap() in holo_kernels.cuh.
struct PlaneDesc {
  float mt_hi, mt_lo;   // m~_j = mt_hi + mt_lo
  float ty, tx;         // sample shift t_kj (pixels), (y, x)
  int by0, bys;         // box rows
  int bx0, bxs;         // box columns
};

// Bilinear tap of one P-grid position along one axis (reading R4): psi index i0 with
// weight 1 - f and i0 + 1 with weight f (taps outside [0, n) are dropped by the user).
// Built in FP64 on the host from xi = m~ (X - P/2) - t + n/2.
struct Tap {
  int i0;
  float f;
};

// Transpose of the taps along one axis: psi index i receives from the P-grid positions
// X0 (weight w0) and X0 + 1 (weight w1); absent contributions have weight 0.
struct AdjTap {
  int X0;
  float w0, w1;
  int pad;
};

// Generic line D-step over rows or columns of a strided complex array.
// The line's nonzero input occupies P-grid positions [in_lo, in_lo + in_len) and is
// read from in[line_in_base + (pos - in_lo) * in_step]; outside, the input is zero.
// The output is written for positions [out_lo, out_lo + out_len) to
// out[line_out_base + (pos - out_lo) * out_step], as out = alpha * D + beta * out.
struct LineArgs {
  const float2* in;
  float2* out;
  long long in_line_stride, in_step;     // element offsets
  long long out_line_stride, out_step;
  int nlines;
  int in_lo, in_len, out_lo, out_len;
  const float2* chirp;                   // P entries, exp(-i pi lambda z f^2) / P
  int conj_chirp;                        // 1: multiply by conj(chirp) (distance -z)
  float alpha;
  int accumulate;                        // 1: out += alpha * D(...)
};

// The column stage of sum_s D_s(x_s) over several sources whose row stage already ran: per
// column of the P x P grid, the transforms of the sources' columns times their chirps are
// summed and transformed back once (see k_cols_sum).
constexpr int kMaxSumSources = 1 + HOLO_MAX_DIST;
struct SumArgs {
  int S;                                     // sources, 1 .. kMaxSumSources
  const float2* in[kMaxSumSources];          // source s: rows [r_lo, r_lo + rows) of the grid,
  int r_lo[kMaxSumSources];                  //   stored [rows][P]
  int rows[kMaxSumSources];
  const float2* chirp[kMaxSumSources];       // P entries, exp(-i pi lambda z_s f^2) / P
  int conj_chirp;                            // 1: conj(chirp) (distance -z_s)
  float alpha;
  int accumulate;                            // 1: out += alpha * sum, else out = alpha * sum
  float2* out;                               // [P][P]
};

// Parameters of the per-plane passes of one forward / gradient evaluation.
struct PassArgs {
  int n, P, J;
  int k0, nk;                  // chunk: global angles [k0, k0 + nk)
  float ext;
  const PlaneDesc* planes;     // [n_angles][J] (global k)
  const float2* psi;           // [nk][n][n]
  const float2* pj;            // [J][P][P]  probe at the sample planes
  const float2* bref;          // [n][n]    C D_{zeta_0}(q)
  // data amplitudes in pass B's column-blocked layout [.][J][dgroups][n][C] (C = the pass-B
  // column-group width): the C columns of a group are contiguous per row, so a warp's loads of
  // consecutive rows of a group are one contiguous run.  Angle k is stored at index k - data_k0.
  const float* dblk;
  int dgroups;
  int data_k0;
  const float2* chirp_zhat;    // [J][P]
  float2* ybuf;                // per local plane: [ystride] (box rows x n)
  long long ystride;
  float2* tq;                  // [n][n]: ext sum_kj r_kj + w_ref r_ref (gradient only)
  int tq_accumulate;           // add to tq instead of overwriting (later parts of a chunk)
  int pb_split;                // pass B: last round split by planes (k_pass_b_split)
  float2* tpart;               // ... its partial S: per block tslots slots of [n][C]
  int tslots;
  int functional;              // 0: F2 (amplitudes, Eq. min1), 1: F1 (intensities, Eq. min2)
  const float2* rref;          // [n][n] reference residual, or null
  float wref;
  float2* gkbuf;               // per local plane: [gkstride] conj(w) v on the box
  long long gkstride;
  float2* u_out;               // optional [nk][J][n][n]
  double* loss_part;           // per block of pass B
  float2* grad_psi;            // [nk][n][n]
  // Dai-Yuan inner products formed by pass D (null: none): Re <g, g> and Re <g, dy_eta> of
  // the grad_psi it writes, one FP64 partial per psi row, at dy_part[kl n + i] and
  // dy_part[nk n + kl n + i]
  const float2* dy_eta;        // [nk][n][n]
  double* dy_part;
  int accumulate;
  const float2* twiddles;      // device twiddle table for this P
  int max_box_rows;            // largest box height of the chunk
  // tap tables of every plane (global index k * J + j)
  const Tap* xtap;             // [planes][tap_stride]: columns [bx0, bx0 + bxs)
  const Tap* ytap;             // [planes][tap_stride]: rows [by0, by0 + bys)
  const AdjTap* xadj;          // [planes][n]: columns of psi
  const AdjTap* yadj;          // [planes][n]: rows of psi
  int tap_stride;
  // rows of all planes in one flat list (plane p owns a contiguous run of its box rows):
  // line -> {global plane, row within the plane's box}
  const int2* lines;           // [total box rows of all planes]
  int line0, nlines;           // the chunk's lines: [line0, line0 + nlines)
  int pass_b_items;            // column groups of pass B
  int pb_blocks;               // pass-B grid of this problem (items of k_pass_b_multi)
  int row_per_sm;              // row passes: resident blocks per SM (0: as many as fit)
  // pass B stages each plane's Y tile [box rows][C columns] into shared memory by TMA
  // while the previous plane computes: tensor map over ybuf as a [planes * yrows][2n] float
  // matrix (box 2C x kStageBox), or null for plain loads
  const void* ymap;
  int yrows;                   // rows per plane in ybuf (ystride / n)
  unsigned long long* err;     // device word, set when a bounded device wait gave up
  // probe shifts (SHIFT forms of passes A-C): per global plane the phase ramps
  // exp(-2 pi i k s / P) of the row (x) and column (y) frequencies k, [planes][P] each;
  // null without probe shifts
  const float2* ramp_x;
  const float2* ramp_y;
};

// Rows of one TMA box of pass B's Y stage (the tensor-map box limit is 256).
constexpr int kStageBox = 256;

// Entry points implemented once per supported line length P.
struct Ops {
  int P;
  cudaError_t (*rows)(const LineArgs&, const float2* tw, cudaStream_t);
  cudaError_t (*cols)(const LineArgs&, const float2* tw, cudaStream_t);
  cudaError_t (*pass_a)(const PassArgs&, cudaStream_t);
  cudaError_t (*pass_b)(const PassArgs&, int with_adjoint, int nblocks, cudaStream_t);
  cudaError_t (*pass_c)(const PassArgs&, cudaStream_t);
  int (*pass_b_groups)(int n);              // column groups of pass B for side n
  int (*pass_b_blocks)(int items, int n, int rows);  // persistent grid of pass B
  int (*pass_b_blocks_split)(long long items, int n);  // ... of its plane-split form
  int (*pass_b_stage_ok)(int n, int rows);  // 1: pass B may stage Y tiles of `rows` rows
  int twiddle_count;
  int pass_b_cols;                          // columns per pass-B group (C)
  int row_lines;                            // lines per block of the row passes (G)
  // several problems of this line length in one persistent launch (args, items in device
  // memory; see k_pass_a_multi / k_pass_b_multi / k_pass_c_multi).  per_sm caps the resident
  // blocks per SM (0: as many as fit); max_n / max_rows size the shared memory for the
  // largest problem.
  cudaError_t (*rows_multi)(int pass_c, const PassArgs* args, const int2* items, int nitems,
                            int shift, int max_n, int per_sm, cudaStream_t);
  cudaError_t (*pass_b_multi)(const PassArgs* args, const int2* items, int nitems, int nprob,
                              int adj, int shift, int max_n, int max_rows, int per_sm,
                              cudaStream_t);
  // the summed column stage (k_cols_sum) and the most sources whose chirps fit its shared
  // memory on the current device
  cudaError_t (*cols_sum)(const SumArgs&, const float2* tw, cudaStream_t);
  int (*cols_sum_max)();
};

const Ops* ops_for(int P);

// Line-length independent kernels (holo_common.cu).
cudaError_t launch_pass_d(const PassArgs& a, cudaStream_t s);
// eta = -g + beta eta, x += gamma eta (as launch_direction_step) with Re <g, eta> of the new
// eta: FP64 partials, one per block, at part[0 .. *nblocks)
cudaError_t launch_direction_step_dot(float2* x, float2* eta, const float2* g, float beta,
                                      float gamma, long long n, double* part, int* nblocks,
                                      cudaStream_t s);
cudaError_t launch_pass_d_multi(const PassArgs* args, const int2* items, int nitems, int nblocks,
                                cudaStream_t s);
// G'_j of the chunk on the box [row0, row0 + nrows) x [col0, col0 + ncols) of the P grid,
// written (or with accumulate added) to out[(Y - orow0) * opitch + (X - ocol0)].
cudaError_t launch_reduce_g(const PassArgs& a, float2* out, int j, int row0, int nrows, int col0,
                            int ncols, int opitch, int orow0, int ocol0, int accumulate,
                            cudaStream_t s);
cudaError_t launch_ref_residual(const float2* bref, const float* sqrt_dref, long long n2,
                                float2* rref, double* part, int nblocks, int functional,
                                cudaStream_t s);
cudaError_t launch_embed_edge(const float* a, int n, int P, float2* q, cudaStream_t s);
cudaError_t launch_block_data(const float* in, long long planes, int n, int C, float* out,
                              cudaStream_t s);
cudaError_t launch_bin_amplitudes(const float* in, long long count, int n, int b, float* out,
                                  cudaStream_t s);
cudaError_t launch_upsample2(const float2* in, long long count, int N, float2* out,
                             cudaStream_t s);
cudaError_t launch_sum_f64(const double* part, int count, double* out, int accumulate,
                           cudaStream_t s);
cudaError_t launch_loss_total(double* red, double wref, int acc, int first, cudaStream_t s);
cudaError_t launch_dot(const float2* a, const float2* b, long long n, double* part, int nblocks,
                       cudaStream_t s);
cudaError_t launch_dot3(const float2* g, const float2* gp, const float2* eta, long long n,
                        double* part, int nblocks, cudaStream_t s);
cudaError_t launch_direction_step(float2* x, float2* eta, const float2* g, float beta, float gamma,
                                  long long n, cudaStream_t s);
cudaError_t launch_axpy(float2* x, const float2* eta, float gamma, long long n, cudaStream_t s);
cudaError_t launch_direction(float2* eta, const float2* g, float beta, long long n,
                             cudaStream_t s);
cudaError_t launch_scale_add(float2* out, const float2* in, float alpha, long long n,
                             int accumulate, cudaStream_t s);
cudaError_t launch_fill_zero(float2* out, long long n, cudaStream_t s);

}  // namespace holo
