// Internal declarations shared by the translation units of libgbi.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gbi.h"

namespace gbi {

constexpr double kPi = 3.14159265358979323846;
// components per sphere of the largest truncation (l <= 5: 83), rounded up; sizes the
// per-component tables passed to kernels by value
constexpr int kMaxD = 84;
// truncations whose pair passes exist in FP64 only: l <= 5 and the minimal set (code 40)
inline bool fp64_only(int trunc) { return trunc == 5 || trunc == 40; }

// Position layouts built once per call from the caller's [N][3] doubles:
//   hi[n] = (float)R, lo[n] = (float)(R - hi)   -> rho = (hi_n - hi_m) + (lo_n - lo_m) in FP32
//   p64[n] = R as double4                        -> FP64 kernels
struct __align__(32) dpos4 {
  double x, y, z, w;
};

struct Positions {
  const float4* hi;
  const float4* lo;
  const dpos4* p64;
};

// Which components a pair pass reads (cols) and writes (rows).
// SET_P (rows only): the 1s rows of a point target of radius zero (flow field evaluation).
enum CompSet : int { SET_ALL = 0, SET_L = 1, SET_H = 2, SET_P = 3 };

struct PairArgs {
  int N;
  double a;
  Positions pos;
  const double* x;       // component-major, first component of the column set
  // FP32 and double-float passes read x as per-sphere source records: sphere m owns
  // rec_floats(NC, df) floats at x32 + m * rec_floats, holding float(x * colscale)
  // padded to a multiple of 4 (double-float: that hi block, then the lo block
  // float(x * colscale - hi)).  The FP64 pass reads x itself.
  const float* x32;
  double* y;             // component-major, first component of the row set
  double alpha, beta;
  int add_self;
  double colscale[kMaxD];   // per-column multiplier applied to x (preconditioner / unit scaling)
  double selfg[kMaxD];    // one-body self scalars g (units 1/a) per component, for add_self
  unsigned int* min_r2_bits;   // optional: atomicMin of the smallest r^2 (float bits), may be null
  // device-side indexing (GMRES on the device): if x_index is set, the kernel reads
  // x + (*x_index) * x_stride; if active is set and *active == 0 the pass does nothing
  const int* x_index;
  size_t x_stride;
  const int* active;
  // batches of independent suspensions: sphere n belongs to system sys_of[n], whose
  // spheres are [sys_off[s], sys_off[s+1]); only those are its sources.  If sys_flag is
  // set, targets of a system with sys_flag[s * sys_flag_stride] == 0 are skipped.
  const int* sys_of;
  const int* sys_off;
  const int* sys_flag;
  int sys_flag_stride;
  int nsys;              // systems in the batch (<= 1: every target's sources are [0, N))
  long long npairs;      // ordered pairs the pass evaluates, for the flop accounting (0: N(N-1))
  int wpt;               // warps per target of the FP32 / double-float kernel (0: default;
                         // 1: the tiled form of pair_tile.cuh, single systems only)
  int pdl;               // launch with programmatic dependent launch (see launch_pdl)
  // tiled form: partial row blocks, one arrival counter per group of 32 targets (zero
  // between launches), the plan (blocks, groups, partial slots per block), the word that
  // records a stage wait that gave up, and the limit of that wait in try_wait rounds
  void* tile_part;
  unsigned int* tile_cnt;
  int tile_P, tile_G, tile_maxseg;
  int* err;
  long long wait_limit;
  // streaming form, single system: targets [split_from, N) (the last, partly filled wave of
  // blocks) have their sources split over nsplit blocks each; each part writes its rows to
  // tile_part (doubles, 32-row chunks) and the last to arrive (tile_cnt, one counter per
  // split target, zero between launches) adds the parts in part order and stores
  int split_from, nsplit;
};

// Programmatic dependent launch: with pdl set the kernel's blocks may be scheduled while
// the previous kernel in the stream is still finishing (its launch latency overlaps that
// kernel's last blocks).  Every kernel launched this way starts with pdl_wait(), which
// returns once all the previous kernel's memory operations are visible, so only block
// scheduling overlaps, never computation.
template <typename... K, typename... A>
inline cudaError_t launch_pdl_smem(bool pdl, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   void (*kernel)(K...), A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}
template <typename... K, typename... A>
inline cudaError_t launch_pdl(bool pdl, dim3 grid, dim3 block, cudaStream_t st, void (*kernel)(K...), A&&... args) {
  return launch_pdl_smem(pdl, grid, block, 0, st, kernel, static_cast<A&&>(args)...);
}

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Floats per source record of a pass reading NC columns (see PairArgs::x32).
inline int rec_floats(int nc, bool df) { return ((nc + 3) & ~3) * (df ? 2 : 1); }

// Largest warps-per-target of the FP32 / double-float pair kernel: a 512-thread block
// would cap the heavier forms (l <= 4, double-float) at 128 registers and spill.
inline int max_wpt(int trunc, int precision) { return (trunc == 4 || precision == 2) ? 8 : 16; }

// Code of the tiled form of pair_tile.cuh (lanes are targets; single systems only).
constexpr int kFormTile = 1;
constexpr int kFormChunk = 3;   // chunk-balanced streaming form (pair_chunk.cuh), one system
inline bool balanced_form(int w) { return w == kFormTile || w == kFormChunk; }

// Warps per target of the FP32 / double-float pair kernel: the requested value (2, 4,
// 8 or 16; 1 selects the tiled form and 3 the chunk-balanced streaming form, which
// serve one system only), else
// enough warps to cover 152 SMs at small N and fewer (less reduction work per target)
// once the N targets alone fill the GPU; capped by max_wpt.
inline int stream_wpt(int trunc, int precision, int N, int requested, bool batched = false) {
  const int d = N >= 8192 ? 2 : (N >= 4096 ? 4 : (N >= 1024 ? 8 : 16));
  if (balanced_form(requested) && !batched && N > 1) return requested;
  const int w = (requested > 1 && !balanced_form(requested)) ? requested : d;
  const int cap = max_wpt(trunc, precision);
  return w < cap ? w : cap;
}

// Launch the generic single-layer pair operator; returns a CUDA error code.
cudaError_t launch_pairs(int trunc, int rows, int cols, int precision, const PairArgs& args,
                         cudaStream_t stream);

struct TrapArgs {
  int N;
  double a, eta;
  Positions pos;
  // per-source data, FP64 from the caller, converted inside the kernel
  const double* Fe;     // [N][3]
  const double* Te;     // [N][3]
  const double* VH;     // [N][h] packed, h = 8 (2s then 3t)
  const double* Va;     // [N][3]
  const double* Oa;     // [N][3]
  double* V;            // [N][3]
  double* Om;           // [N][3]
};

// Three launches (record packing, split pair sums, fixed-order reduction); scratch must
// hold trap_scratch_bytes(N, precision) bytes, 256-byte aligned.
cudaError_t launch_trap(const TrapArgs& args, int precision, void* scratch, cudaStream_t stream);
size_t trap_scratch_bytes(int N, int precision);
int trap_splits(int N, int precision);

// Learned near-field correction (mlp_kernel.cu).  Layout and definitions: gbi.h.
namespace mlpk {
#ifdef __CUDACC__
// tanh of the inference kernels: the hardware approximation (PTX tanh.approx.f32, relative
// error about 2^-11), below the bf16 rounding that every activation receives next
__device__ __forceinline__ float tanh_act(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
#endif
constexpr int NIN = 9, NH = 128, NOUT = 6;
constexpr int NPARAM = NH * NIN + NH + 2 * (NH * NH + NH) + NOUT * NH + NOUT;   // 35078
// What the six outputs of a pair are (gbi_mlp_set_head): 0 = the velocity and angular
// velocity corrections of the target (two vectors in the pair frame); 1 = the correction
// of its strain-mode flow coefficient Q^(2s) (outputs 0..4: the packed symmetric
// traceless tensor in the pair frame; output 5 is trained toward zero and not used).
constexpr int HEAD_VELOCITY = 0, HEAD_QSTRAIN = 1;
#ifdef __CUDACC__
// Packed coordinates of a symmetric traceless 3x3 tensor in the orthonormal basis of the
// mode layout (components sqrt2 xy, sqrt2 yz, (2zz - xx - yy)/sqrt6, sqrt2 xz, (xx - yy)/sqrt2).
__device__ __forceinline__ void stf2_unpack(const float* q, float S[3][3]) {
  const float r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
  S[0][0] = -r6 * q[2] + r2 * q[4];
  S[1][1] = -r6 * q[2] - r2 * q[4];
  S[2][2] = 2.0f * r6 * q[2];
  S[0][1] = S[1][0] = r2 * q[0];
  S[1][2] = S[2][1] = r2 * q[1];
  S[0][2] = S[2][0] = r2 * q[3];
}
__device__ __forceinline__ void stf2_pack(const float T[3][3], float* q) {
  const float s2 = 1.41421356237309505f, r2 = 0.70710678118654752f, r6 = 0.40824829046386302f;
  q[0] = s2 * T[0][1];
  q[1] = s2 * T[1][2];
  q[2] = r6 * (2.0f * T[2][2] - T[0][0] - T[1][1]);
  q[3] = s2 * T[0][2];
  q[4] = r2 * (T[0][0] - T[1][1]);
}
// The rank-2 tensor with pair-frame coordinates q, in lab coordinates (to_lab: sum_kl
// S_kl e_k e_l), or the lab tensor q in pair-frame coordinates (e_k . S . e_l).  fr holds
// the rows e_x, e_y, e_z.
__device__ __forceinline__ void stf2_rotate(const float* fr, const float* q, float* out, bool to_lab) {
  float S[3][3], T[3][3];
  stf2_unpack(q, S);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = 0; l < 3; ++l) {
          const float a = to_lab ? fr[3 * k + i] : fr[3 * i + k];
          const float b = to_lab ? fr[3 * l + j] : fr[3 * j + l];
          acc = fmaf(a * b, S[k][l], acc);
        }
      T[i][j] = acc;
    }
  stf2_pack(T, out);
}
// Lab-frame per-pair contribution dst[6] from the pair-frame outputs y[6].
__device__ __forceinline__ void pair_out_to_lab(int head, const float* fr, const float* y, float* dst) {
  if (head == HEAD_QSTRAIN) {
    stf2_rotate(fr, y, dst, true);
    dst[5] = y[5];
    return;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dst[i] = y[0] * fr[i] + y[1] * fr[3 + i] + y[2] * fr[6 + i];
    dst[3 + i] = y[3] * fr[i] + y[4] * fr[3 + i] + y[5] * fr[6 + i];
  }
}
// Gradient with respect to the pair-frame outputs from the gradient dp[6] with respect to
// the lab-frame contribution (the transpose of pair_out_to_lab, itself orthogonal).
__device__ __forceinline__ void lab_grad_to_pair(int head, const float* fr, const float* dp, float* g) {
  if (head == HEAD_QSTRAIN) {
    stf2_rotate(fr, dp, g, false);
    g[5] = dp[5];
    return;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g[c] = fr[3 * c] * dp[0] + fr[3 * c + 1] * dp[1] + fr[3 * c + 2] * dp[2];
    g[3 + c] = fr[3 * c] * dp[3] + fr[3 * c + 1] * dp[4] + fr[3 * c + 2] * dp[5];
  }
}
#endif
size_t scan_scratch_ints(int n);
cudaError_t exclusive_scan(const int* in, int* out, int n, int* scratch, cudaStream_t st);
cudaError_t bbox(int N, const double* R, double* part_dev, double* out_host, cudaStream_t st);
cudaError_t nb_count_sys(int N, const double* R, const int* sys_of, const int* sys_off, double rc2, int* cnt,
                         cudaStream_t st);
cudaError_t nb_fill_sys(int N, const double* R, const int* sys_of, const int* sys_off, double rc2, const int* start,
                        int* tg, int* sr, cudaStream_t st);
cudaError_t cells_build(int N, const double* R, const double* box, double side, int* dims, int* cell_of,
                        int* cell_cnt, int* cell_start, int* cell_fill, int* items, int* scratch, cudaStream_t st);
cudaError_t nb_cells(int N, const double* R, const double* box, double side, const int* dims, const int* cell_of,
                     const int* cell_start, const int* cell_cnt, const int* items, double rc2, const int* start,
                     int* cnt, int* tg, int* sr, int* overflow, cudaStream_t st);
cudaError_t features(int P, const double* R, const double* p, const int* tg, const int* sr, double a, float* F,
                     float* FR, cudaStream_t st);
size_t packed_bytes();
cudaError_t pack_weights(const float* theta, float* thq, void* packed, cudaStream_t st);
cudaError_t infer(int P, const float* F, const float* FR, const void* packed, float* out, int num_sms, int head,
                  cudaStream_t st);
cudaError_t sphere_sums(int N, const int* start, const float* lab, double scale, double* V, double* Om,
                        cudaStream_t st);
// QH[n][0..4] (rows of h) += scale * the sums of n's pairs' first five outputs
cudaError_t sphere_sums_q(int N, const int* start, const float* lab, double scale, double* QH, int h,
                          cudaStream_t st);
size_t train_part_floats(int max_pairs);
cudaError_t train_batch(const float* thq, const float* F, const float* FR, const int* start, const double* labels,
                        int p_begin, int p_end, int n_begin, int n_end, int ns_total, float* lab, float* dO,
                        float* part, double* loss_part, float* grad, int head, int engine, const void* packed_tc,
                        int* err, int num_sms, cudaStream_t st);
// tensor-core backward of the pairs [0, P) (F, dO already offset): one partial gradient
// per block in part; the number of blocks it uses
cudaError_t train_bwd_tc(int P, const float* F, const float* dO, const void* packed, float* part, int* err,
                         int num_sms, cudaStream_t st);
int train_bwd_tc_blocks(int P, int num_sms);
cudaError_t adam(float* th, float* m, float* v, const float* g, int t, double lr, float* thq, void* packed,
                 void* packed_tc, cudaStream_t st);
cudaError_t sum_into(const double* parts, int n, double* dst, cudaStream_t st);
// tcgen05 inference (mlp_tc.cu): own packed layout; *err is set if a wait gave up
size_t packed_tc_bytes();
cudaError_t pack_weights_tc(const float* theta, void* packed, cudaStream_t st);
cudaError_t infer_tc(int P, const float* F, const float* FR, const void* packed, float* out, int* err, int num_sms,
                     int head, cudaStream_t st);
cudaError_t labels(int N, double s0, double sigma, const double* Vx, const double* Ox, const double* Vs,
                   const double* Os, double* out, double* sq_part, cudaStream_t st);
// labels[n] = sigma / s0 * (QHx - QH1)[n][0..4], 0 (rows of h); block partial sums of squares
cudaError_t labels_q(int N, int h, double s0, double sigma, const double* QHx, const double* QH1, double* out,
                     double* sq_part, cudaStream_t st);
}  // namespace mlpk

// Flop counts per ordered pair used for the roofline accounting.
double pair_flops(int trunc, int rows, int cols);
double trap_flops();

}  // namespace gbi
