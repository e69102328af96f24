// Internal to libgbi: the state behind a gbi_ctx handle and the helpers, small kernels
// and solver entry points that the library's translation units share (common.cu,
// solver.cu, nearfield_api.cu, gbi_api.cu).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "gbi_generated.cuh"
#include "gbi_internal.cuh"

namespace gbi {
// a device buffer of the workspace, grown on demand by ensure()
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};
// nesting depth of the conditional bodies in the solve graph (one capture stream each)
constexpr int kCapLevels = 4;
// classes of gbi_kernel_stats: pair passes 0..26 (precision x 9 + rows x 3 + cols), closed-form
// trap kernel 27 (FP64) / 28 (FP32), flow field 29 / 30, wall images 31 / 32
constexpr int kStatClasses = 33;
}  // namespace gbi

struct gbi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  gbi::Buf pos_hi, pos_lo, pos64;                // centres: hi / lo floats, FP64 copy
  gbi::Buf b, xQ, r, delta, krylov, w, xVL, minr2, x32, trapbuf, gstate;   // solve workspace
  gbi::Buf boff, bsys;                           // system offsets / ids of the current batch
  gbi::Buf tile, tilecnt;                        // tiled pair passes: partial sums, arrival counters
  gbi::Buf flowx, flowrec, flowcnt;              // gbi_flow: coefficients, FP32 records, inside count
  gbi::Buf wallbuf;                              // gbi_wall_superpose: source records and slice partials
  gbi::Buf perbuf;                               // gbi_periodic_superpose: records, cells, wave vectors, S(k)
  long long wait_limit = 1ll << 24;              // try_wait rounds of a tiled pass's stage waits
                                                 // (kTileWaitLimit; gbi_set_wait_limit)
  int single_N = -1;                             // boff / bsys hold one system of this many spheres
  const void* single_off = nullptr;              // ... in these buffers
  const void* single_sys = nullptr;
  int single_off_host[2] = {0, 0};               // source of that upload (outlives the async copy)
  char* hs = nullptr;                            // host scratch: per-system solver states, counters
  size_t hs_cap = 0;
  std::vector<char> hs_own;                      // its storage (a static array for gbi_solve_static)
  bool allow_graphs = true;                      // run each GMRES cycle as one CUDA graph
  bool fixed = false;                            // buffers bound to static storage: never reallocate
  cudaGraphExec_t chunk_exec = nullptr;          // device-looped Arnoldi steps of one GMRES cycle
  const void* chunk_key[8] = {};                 // buffers and sizes the graph was built for
  long long chunk_ikey[6] = {};
  int chunk_nodes = 0;                           // kernels per loop iteration
  // the whole mixed-precision solve as one graph: built when a call repeats the previous
  // call's key (buffers, sizes, parameters, tuning), replayed while the key stays
  cudaGraphExec_t solve_exec = nullptr;
  std::vector<long long> solve_key, solve_prev, solve_failed;
  long long solve_own[5] = {};                   // kernels: top level, per sweep, inner solve, cycle, step
  cudaStream_t cap[gbi::kCapLevels] = {};        // capture streams of the nested bodies
  gbi::Buf dsolve;                               // its device-side counters
  long long wpt_gen = 0;                         // bumped whenever the warps-per-target choice changes
  long long solve_replays = 0;                   // solves run from solve_exec
  bool pdl = true;                               // programmatic dependent launch in the Arnoldi steps
  gbi::Buf tFe, tTe, tVa, tOa, tVH, tV, tOm, tQH;  // trap-step staging
  int tqh_N = -1, tqh_trunc = -1;                // tQH holds the last trap-step solution of this size
  gbi::Buf hR, hVa, hOa, hVH, hFe, hTe, hV, hOm, hQH;  // gbi_solve_host staging
  long long launches = 0;                        // kernels launched by this context
  bool prof = false;                             // record events around pair passes
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    double flops;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double stat_ms[gbi::kStatClasses] = {0};
  double stat_flops[gbi::kStatClasses] = {0};
  long long stat_n[gbi::kStatClasses] = {0};
  long long stat_dead[gbi::kStatClasses] = {0};
  // learned near-field correction: FP32 master weights, Adam moments, bf16-rounded
  // copy (training), padded bf16 copy (inference), gradient; neighbour lists; pair
  // features, outputs and training scratch
  gbi::Buf mlp_th, mlp_m, mlp_v, mlp_thq, mlp_pk, mlp_grad, mlp_pk_tc, mlp_err;
  int split_tail = 0;                            // split the streaming pass's partly filled last wave
  int mlp_engine = 1;                            // inference: 0 mma.sync, 1 tcgen05
  int mlp_head = 0;                              // what the outputs are (mlpk::HEAD_*)
  double mlp_sigma = 0.0;
  int mlp_step = 0;
  bool mlp_ready = false;
  gbi::Buf nb_cnt, nb_start, nb_tg, nb_sr, nb_scan, cell_of, cell_cnt, cell_start, cell_fill, cell_items, nb_aux;
  int nb_pairs = 0, nb_N = 0;
  gbi::Buf mf_F, mf_FR, mf_lab, mf_dO, mf_part, mf_loss;
  int num_sms = 0;
  // warps per target chosen by gbi_tune, keyed by pass, precision, log2(N), batching
  std::map<long long, int> wpt_table;
  int force_wpt = 0;                             // gbi_set_wpt override (0: table or default)
  static long long wpt_key(int trunc, int rows, int cols, int precision, int N, bool batched) {
    int lg = 0;
    while (lg < 40 && (2LL << lg) <= N) ++lg;
    return ((((long long)(trunc * 3 + rows) * 3 + cols) * 3 + precision) * 64 + lg) * 2 + (batched ? 1 : 0);
  }
  int tuned_wpt(int trunc, int rows, int cols, int precision, int N, bool batched) const {
    const auto it = wpt_table.find(wpt_key(trunc, rows, cols, precision, N, batched));
    return it == wpt_table.end() ? 0 : it->second;
  }
};

namespace gbi {

constexpr int kMaxRestart = 128;   // GMRES restart length cap (Krylov vectors per cycle)
constexpr int kFusedBlocks = 64;   // blocks of the fused single-system Arnoldi step

// CUDA error -> status, keeping the message in the context
gbi_status fail(gbi_ctx* c, cudaError_t e, const char* where);

#define GBI_CHECK(call)                                           \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) return fail(ctx, e_, #call);           \
  } while (0)

#define GBI_TRY(call)                      \
  do {                                     \
    gbi_status s_ = (call);                \
    if (s_ != GBI_OK) return s_;           \
  } while (0)

// at least `bytes` of host scratch in ctx->hs (never shrinks; refuses for static storage)
gbi_status host_scratch(gbi_ctx* ctx, size_t bytes);
// grow a workspace buffer to at least `bytes` (never shrinks; refuses for static storage)
gbi_status ensure(gbi_ctx* ctx, Buf& b, size_t bytes);
template <typename T> T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

cudaEvent_t take_event(gbi_ctx* ctx);
int sm_count(gbi_ctx* ctx);
// Resolve recorded event pairs into per-class totals (blocks on the last one).
void drain_profile(gbi_ctx* ctx);

// One pair pass with launch counting and optional event timing.
// Class: precision * 9 + rows * 3 + cols for the generic operator (precision 0 FP64,
// 1 FP32, 2 double-float), 27/28 for the closed-form trap kernel in FP64/FP32, 29/30 for
// the flow-field kernel in FP64/FP32.
template <typename F>
cudaError_t timed(gbi_ctx* ctx, int cls, double flops, int nlaunch, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (ctx->prof) {
    a = take_event(ctx);
    b = take_event(ctx);
    cudaEventRecord(a, ctx->stream);
  }
  cudaError_t e = launch();
  ctx->launches += nlaunch;
  if (ctx->prof) {
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({a, b, cls, flops});
  }
  return e;
}

struct ColScale {
  double v[kMaxD];
};

cudaError_t launch_records(bool dfl, int N, int nc, const double* x, const int* xi, size_t xs, const int* active,
                           const ColScale& cs, float* rec, cudaStream_t stream);
int ncols_of(int trunc, int cols);
cudaError_t run_pairs(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, const PairArgs& args_in);
// ctx->minr2 holds four words: [0] smallest r^2 (float bits) of the overlap guard, [1] set
// by a tiled pair pass whose stage wait gave up, [2] non-finite solve input.  Allocated
// (cleared) on first use.
gbi_status status_words(gbi_ctx* ctx);
int* pass_error_word(gbi_ctx* ctx);
// [2]: set by the input-packing kernels of a solve when an input is NaN or infinite
int* input_error_word(gbi_ctx* ctx);
// clear the error word and the tiled passes' counters after a pass gave up
gbi_status pass_error_reset(gbi_ctx* ctx);
struct TilePlan;
// scratch of a tiled pass over N spheres with these rows in this precision
gbi_status tile_reserve(gbi_ctx* ctx, int trunc, int rows, int precision, int N, TilePlan* out);
// plan and scratch of the balanced form a.wpt (tiled or chunk-balanced) for a pass over N
// spheres, into a; false if the scratch cannot be had
bool balanced_args(gbi_ctx* ctx, int trunc, int rows, int precision, int N, PairArgs& a);
// the split of the streaming form's partly filled last wave (split_from, nsplit of
// PairArgs) and its scratch in the context; false (and no split) if it does not pay or its
// scratch cannot be had
bool split_reserve(gbi_ctx* ctx, int trunc, int rows, int precision, PairArgs& a);
cudaError_t run_trap(gbi_ctx* ctx, const TrapArgs& t, int precision);
int d_of(int trunc);
const double* scale_tab(int trunc);
const double* self_tab(int trunc);

struct Scales {
  double v[kMaxD];
};

__global__ void k_pack_lower(int N, double a, double c2a, const double* __restrict__ Fe,
                             const double* __restrict__ Te, double* xF, int* bad);
__global__ void k_pack_higher(int N, int h, const double* __restrict__ VH, Scales sc, double mult,
                              double* out, int* bad);
__global__ void k_unpack_higher(int N, int h, const double* __restrict__ x, Scales sc, double* QH);
__global__ void k_finalize_lower(int N, double a, double c2a, const double* __restrict__ xVL,
                                 const double* __restrict__ Va, const double* __restrict__ Oa,
                                 double* V, double* Om, int* bad);

inline unsigned grid1(size_t n, int bs = 256) { return unsigned((n + bs - 1) / bs); }

// solver state for one call
struct Setup {
  int N, trunc, D, h;
  double a, eta;
  Scales scale;     // internal scale per component (all D)
  Scales selfg;     // self scalars per component (units 1/a)
  Scales minv;      // H components: a / g (right Jacobi preconditioner)
  Scales ones;
  Positions pos;
  long long pairs_per_pass;
};

gbi_status setup_call(gbi_ctx* ctx, Setup& s, int N, int trunc, double a, double eta, const double* R,
                      bool launch_positions = true);
// the centres of R as float hi / lo and FP64 copies (what setup_call launches)
gbi_status launch_positions(gbi_ctx* ctx, const Setup& s, const double* R, int* bad = nullptr);
PairArgs pair_args(const Setup& s, const double* x, double* y, double alpha, double beta, int add_self,
                   const Scales& colscale, int col0);

// Independent systems of one batched call: system s holds spheres [off[s], off[s+1]).
struct Batch {
  int S = 1;
  int Ntot = 0;
  const int* off = nullptr;   // device [S+1]
  const int* sys = nullptr;   // device [Ntot]
  const int* h_off = nullptr; // host copy of off (the caller's array, or one[] below)
  int one[2] = {0, 0};        // offsets of the single-system case
  Batch() = default;
  Batch(const Batch&) = delete;   // h_off may point into the object
  Batch& operator=(const Batch&) = delete;
};

bool valid_params(const gbi_params* p);
// ordered pairs of a batch, sum over its systems of n (n - 1)
long long batch_pairs(const Batch& B);
bool valid_offsets(int nsys, const int* off);
gbi_status make_batch(gbi_ctx* ctx, int nsys, const int* offsets_host, Batch& B);
gbi_status single_batch(gbi_ctx* ctx, int N, Batch& B);
// Counters of the device-decided solve (one record per call, read back at the end):
// what the host-driven sequence accumulates in gbi_info, plus the number of times each
// loop body of the solve graph ran.
struct DSolve {
  long long iters;        // inner GMRES iterations over the whole solve
  long long mv32, mv64;   // pair passes decided on the device
  long long pairs;        // their ordered pairs
  long long steps;        // Arnoldi loop iterations
  long long cycles;       // GMRES cycles
  int refinements;        // refinement sweeps after the first
  int ifs;                // sweeps that ran an inner solve
  int first, notfirst;    // the current inner solve is in its first cycle / past it
  int overlap;            // the overlap guard stopped the solve
  int bad_input;          // an input was NaN or infinite: the solve stopped
  double rel_max;         // largest final relative residual over the systems
};

// Work a caller wraps around one solve (a trap step: the inputs from (R, p) before, the
// Euler update after).  solve_core launches `before` ahead of its own packing and `after`
// once the solve has succeeded; in a replayed solve graph both are captured with the solve
// (the caller's arrays then belong to the graph's key) and `after` receives the device
// record, so that its kernels can skip the update of a solve that failed.
struct StepHooks {
  std::function<gbi_status()> before;
  std::function<gbi_status(const DSolve* rec)> after;   // rec: device record, or null
  std::vector<long long> key;                           // values the hooks' launches depend on
};

gbi_status solve_core(gbi_ctx* ctx, const gbi_params* prm, const Batch& B, const double* R, const double* Va,
                      const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                      double* Omega, double* QH, int warm_start, gbi_info* inf, const StepHooks* hooks = nullptr);

}  // namespace gbi
