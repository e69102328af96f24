// C ABI of libgbi: context, workspace, input/output packing, GMRES with FP64 Arnoldi
// and Givens least squares, mixed-precision iterative refinement, superposition and
// the harmonic-trap integrator.  Every arithmetic step of the method runs in the
// kernels of this library; the host only sequences launches and runs the
// (m+1) x m Givens/triangular solve of GMRES on scalars read back from the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "gbi_generated.cuh"
#include "gbi_internal.cuh"

namespace gbi {
#define GBI_DECL(P)                                                                       \
  cudaError_t launch_pairs_##P##_2(int, int, const PairArgs&, cudaStream_t);              \
  cudaError_t launch_pairs_##P##_3(int, int, const PairArgs&, cudaStream_t);              \
  cudaError_t launch_pairs_##P##_4(int, int, const PairArgs&, cudaStream_t);
GBI_DECL(f32)
GBI_DECL(f64)
GBI_DECL(df)
#undef GBI_DECL

// precision: 0 = FP64, 1 = FP32, 2 = double-float on the FP32 pipe
cudaError_t launch_pairs(int trunc, int rows, int cols, int precision, const PairArgs& args,
                         cudaStream_t stream) {
#define GBI_DISPATCH(P)                                                   \
  if (trunc == 2) return launch_pairs_##P##_2(rows, cols, args, stream);  \
  if (trunc == 3) return launch_pairs_##P##_3(rows, cols, args, stream);  \
  if (trunc == 4) return launch_pairs_##P##_4(rows, cols, args, stream);  \
  return cudaErrorInvalidValue;
  if (precision == 1) { GBI_DISPATCH(f32) }
  if (precision == 2) { GBI_DISPATCH(df) }
  GBI_DISPATCH(f64)
#undef GBI_DISPATCH
}

double pair_flops(int trunc, int rows, int cols) {
  if (rows < 0 || rows > 2 || cols < 0 || cols > 2) return 0.0;
  if (trunc == 2) return gbi_t2_flops[rows][cols];
  if (trunc == 3) return gbi_t3_flops[rows][cols];
  if (trunc == 4) return gbi_t4_flops[rows][cols];
  return 0.0;
}
}  // namespace gbi

using namespace gbi;

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct gbi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  Buf pos_hi, pos_lo, pos64;
  Buf xF, xVH, b, xQ, r, delta, krylov, w, partial, dots, xVL, minr2, colbuf, x32, trapbuf, gstate;
  Buf boff, bsys;                              // system offsets / ids of the current batch
  std::vector<char> hbatch;                    // host copy of the per-system solver states
  bool allow_graphs = true;                    // replay Arnoldi chunks from a CUDA graph
  bool fixed = false;                          // buffers bound to static storage: never reallocate
  cudaGraphExec_t chunk_exec = nullptr;        // device-looped Arnoldi steps of one GMRES cycle
  const void* chunk_key[8] = {};
  long long chunk_ikey[6] = {};
  int chunk_nodes = 0;
  Buf tFe, tTe, tVa, tOa, tVH, tV, tOm, tQH;   // trap-step / host-call staging
  int tqh_N = -1, tqh_trunc = -1;              // tQH holds the last trap-step solution of this size
  Buf hR, hVa, hOa, hVH, hFe, hTe, hV, hOm, hQH;
  double* hbuf = nullptr;                      // pinned scalars read back by GMRES
  long long launches = 0;                      // kernels launched by this context
  bool prof = false;                           // record events around pair passes
  struct Rec {
    cudaEvent_t a, b;
    int cls;
    double flops;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double stat_ms[30] = {0};
  double stat_flops[30] = {0};
  long long stat_n[30] = {0};
  long long stat_dead[30] = {0};
  // learned near-field correction: FP32 master weights, Adam moments, bf16-rounded
  // copy (training), padded bf16 copy (inference), gradient; neighbour lists; pair
  // features, outputs and training scratch
  Buf mlp_th, mlp_m, mlp_v, mlp_thq, mlp_pk, mlp_grad, mlp_pk_tc, mlp_err;
  int mlp_engine = 1;                          // inference: 0 mma.sync, 1 tcgen05
  double mlp_sigma = 0.0;
  int mlp_step = 0;
  bool mlp_ready = false;
  Buf nb_cnt, nb_start, nb_tg, nb_sr, nb_scan, cell_of, cell_cnt, cell_start, cell_fill, cell_items, nb_aux;
  int nb_pairs = 0, nb_N = 0;
  Buf mf_F, mf_FR, mf_lab, mf_dO, mf_part, mf_loss;
  int num_sms = 0;
  // warps per target chosen by gbi_tune, keyed by pass, precision, log2(N), batching
  std::map<long long, int> wpt_table;
  int force_wpt = 0;                           // gbi_set_wpt override (0: table or default)
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

namespace {

constexpr int kMaxRestart = 128;

gbi_status fail(gbi_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return GBI_OK;
  c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GBI_ERR_NOMEM : GBI_ERR_CUDA;
}

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

gbi_status ensure(gbi_ctx* ctx, Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return GBI_OK;
  if (ctx->fixed) {
    ctx->err = "static scratch too small for this request";
    return GBI_ERR_NOMEM;
  }
  if (b.p) {
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    GBI_CHECK(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
  }
  GBI_CHECK(cudaMalloc(&b.p, bytes));
  b.bytes = bytes;
  return GBI_OK;
}

template <typename T> T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

cudaEvent_t take_event(gbi_ctx* ctx) {
  if (!ctx->pool.empty()) {
    cudaEvent_t e = ctx->pool.back();
    ctx->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Resolve recorded event pairs into per-class totals (blocks on the last one).
void drain_profile(gbi_ctx* ctx) {
  for (auto& r : ctx->pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    ctx->stat_ms[r.cls] += ms;
    ctx->stat_flops[r.cls] += r.flops;
    ctx->stat_n[r.cls] += 1;
    ctx->pool.push_back(r.a);
    ctx->pool.push_back(r.b);
  }
  ctx->pending.clear();
}

// One pair pass with launch counting and optional event timing.
// Class: precision * 9 + rows * 3 + cols for the generic operator (precision 0 FP64,
// 1 FP32, 2 double-float), 27/28 for the closed-form trap kernel in FP64/FP32.
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
  double v[54];
};

// Source records of the FP32 / double-float passes (see PairArgs::x32): from the
// component-major [nc][N] block x (optionally device-indexed; skipped when the
// device-side solver has stopped), rec[m] = float(x[.][m] * cs) padded with zeros to
// ncp floats (double-float: then the lo block).  One block per 32 spheres, transposed
// through shared memory so that both the reads and the writes are coalesced.
template <bool DFL>
__global__ void k_records(int N, int nc, int ncp, const double* __restrict__ x, const int* xi, size_t xs,
                          const int* active, ColScale cs, float* __restrict__ rec) {
  extern __shared__ float tile[];   // [32][rf + 1]
  if (active != nullptr && *active == 0) return;
  if (xi != nullptr) x += (size_t)(*xi) * xs;
  const int rf = DFL ? 2 * ncp : ncp;
  const int m0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int m = m0 + lane;
  for (int q = wy; q < ncp; q += nw) {
    float h = 0.f, l = 0.f;
    if (q < nc && m < N) {
      const double v = x[(size_t)q * N + m] * cs.v[q];
      h = float(v);
      l = float(v - double(h));
    }
    tile[lane * (rf + 1) + q] = h;
    if (DFL) tile[lane * (rf + 1) + ncp + q] = l;
  }
  __syncthreads();
  const int cnt = min(32, N - m0);
  for (int i = threadIdx.x; i < cnt * rf; i += blockDim.x) {
    const int r = i / rf, c = i - r * rf;
    rec[(size_t)(m0 + r) * rf + c] = tile[r * (rf + 1) + c];
  }
}

cudaError_t launch_records(bool dfl, int N, int nc, const double* x, const int* xi, size_t xs, const int* active,
                           const ColScale& cs, float* rec, cudaStream_t stream) {
  const int ncp = (nc + 3) & ~3;
  const int rf = dfl ? 2 * ncp : ncp;
  const size_t smem = sizeof(float) * 32 * (rf + 1);
  const dim3 grid((N + 31) / 32), block(256);
  if (dfl) k_records<true><<<grid, block, smem, stream>>>(N, nc, ncp, x, xi, xs, active, cs, rec);
  else k_records<false><<<grid, block, smem, stream>>>(N, nc, ncp, x, xi, xs, active, cs, rec);
  return cudaGetLastError();
}

int ncols_of(int trunc, int cols) {
  const int D = trunc == 2 ? GbiTrunc2::D : trunc == 3 ? GbiTrunc3::D : GbiTrunc4::D;
  return cols == SET_L ? 6 : cols == SET_H ? D - 6 : D;
}

cudaError_t run_pairs(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, const PairArgs& args_in) {
  const double flops = pair_flops(trunc, rows, cols) * double(args_in.N) * double(args_in.N - 1);
  PairArgs args = args_in;
  int extra = 0;
  if (args.wpt == 0)
    args.wpt = ctx->force_wpt > 0 ? ctx->force_wpt
                                  : ctx->tuned_wpt(trunc, rows, cols, precision, args.N, args.sys_of != nullptr);
  if (precision == 2 || (precision == 1 && args.x32 == nullptr)) {
    // per-sphere source records (FP32, or the double-float hi/lo pair), once per pass,
    // so that the pair loop touches no FP64
    const int nc = ncols_of(trunc, cols);
    const size_t bytes = sizeof(float) * rec_floats(nc, precision == 2) * (size_t)args.N;
    if (ensure(ctx, ctx->x32, bytes) != GBI_OK) return cudaErrorMemoryAllocation;
    ColScale cs;
    const int c0 = cols == SET_H ? 6 : 0;
    for (int i = 0; i < 54; ++i) cs.v[i] = (i < nc) ? args.colscale[c0 + i] : 1.0;
    const cudaError_t e = launch_records(precision == 2, args.N, nc, args.x, args.x_index, args.x_stride,
                                         args.active, cs, P<float>(ctx->x32), ctx->stream);
    if (e != cudaSuccess) return e;
    args.x32 = P<float>(ctx->x32);
    extra = 1;
  }
  return timed(ctx, precision * 9 + rows * 3 + cols, flops, 1 + extra,
               [&] { return launch_pairs(trunc, rows, cols, precision, args, ctx->stream); });
}

cudaError_t run_trap(gbi_ctx* ctx, const TrapArgs& t, int precision) {
  const double flops = trap_flops() * double(t.N) * double(t.N - 1);
  if (ensure(ctx, ctx->trapbuf, trap_scratch_bytes(t.N, precision)) != GBI_OK) return cudaErrorMemoryAllocation;
  return timed(ctx, precision == 1 ? 28 : 27, flops, 3,
               [&] { return launch_trap(t, precision, ctx->trapbuf.p, ctx->stream); });
}

int d_of(int trunc) { return trunc == 2 ? GbiTrunc2::D : trunc == 3 ? GbiTrunc3::D : trunc == 4 ? GbiTrunc4::D : -1; }
const double* scale_tab(int trunc) { return trunc == 2 ? gbi_t2_scale : trunc == 3 ? gbi_t3_scale : gbi_t4_scale; }
const double* self_tab(int trunc) { return trunc == 2 ? gbi_t2_self : trunc == 3 ? gbi_t3_self : gbi_t4_self; }

// ---------------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------------

__global__ void k_positions(int N, const double* __restrict__ R, float4* hi, float4* lo, dpos4* p64) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double x = R[3 * n], y = R[3 * n + 1], z = R[3 * n + 2];
  const float hx = float(x), hy = float(y), hz = float(z);
  hi[n] = make_float4(hx, hy, hz, 0.f);
  lo[n] = make_float4(float(x - double(hx)), float(y - double(hy)), float(z - double(hz)), 0.f);
  p64[n] = dpos4{x, y, z, 0.0};
}

// F^(1) = -F^e and F^(21) = -T^e/a in internal coordinates: xF[6][N]
__global__ void k_pack_lower(int N, double a, double c2a, const double* __restrict__ Fe,
                             const double* __restrict__ Te, double* xF) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* f = Fe + 3 * n;
  const double* t = Te + 3 * n;
  xF[0 * N + n] = -f[1];
  xF[1 * N + n] = -f[2];
  xF[2 * N + n] = -f[0];
  xF[3 * N + n] = -c2a * t[1] / a;
  xF[4 * N + n] = -c2a * t[2] / a;
  xF[5 * N + n] = -c2a * t[0] / a;
}

struct Scales {
  double v[54];
};

// packed [N][h] -> internal component-major [h][N] times scale * mult
__global__ void k_pack_higher(int N, int h, const double* __restrict__ VH, Scales sc, double mult,
                              double* out) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)N * h) return;
  const int n = int(i / h), p = int(i - (size_t)n * h);
  out[(size_t)p * N + n] = mult * sc.v[p] * VH[i];
}

// internal [h][N] -> packed [N][h] divided by scale
__global__ void k_unpack_higher(int N, int h, const double* __restrict__ x, Scales sc, double* QH) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)N * h) return;
  const int n = int(i / h), p = int(i - (size_t)n * h);
  QH[i] = x[(size_t)p * N + n] / sc.v[p];
}

// V = V^a + (1s part), Omega = Omega^a + (2a part)/(c_2a 2a)
__global__ void k_finalize_lower(int N, double a, double c2a, const double* __restrict__ xVL,
                                 const double* __restrict__ Va, const double* __restrict__ Oa,
                                 double* V, double* Om) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double f = 1.0 / (c2a * 2.0 * a);
  V[3 * n + 0] = Va[3 * n + 0] + xVL[2 * N + n];
  V[3 * n + 1] = Va[3 * n + 1] + xVL[0 * N + n];
  V[3 * n + 2] = Va[3 * n + 2] + xVL[1 * N + n];
  Om[3 * n + 0] = Oa[3 * n + 0] + f * xVL[5 * N + n];
  Om[3 * n + 1] = Oa[3 * n + 1] + f * xVL[3 * N + n];
  Om[3 * n + 2] = Oa[3 * n + 2] + f * xVL[4 * N + n];
}

__global__ void k_trap_inputs(int N, double k_trap, double vs, double s0, double d0, int h,
                              const double* __restrict__ R, const double* __restrict__ p, double* Fe,
                              double* Te, double* Va, double* Oa, double* VH) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double px = p[3 * n], py = p[3 * n + 1], pz = p[3 * n + 2];
  for (int i = 0; i < 3; ++i) {
    Fe[3 * n + i] = -k_trap * R[3 * n + i];
    Te[3 * n + i] = 0.0;
    Oa[3 * n + i] = 0.0;
  }
  Va[3 * n] = vs * px;
  Va[3 * n + 1] = vs * py;
  Va[3 * n + 2] = vs * pz;
  double* vh = VH + (size_t)h * n;
  for (int i = 0; i < h; ++i) vh[i] = 0.0;
  double q[5];
  gbi_pack2<double>(px, py, pz, q);          // U_mu . pp (the -I/3 part is traceless-projected away)
  for (int i = 0; i < 5; ++i) vh[i] = s0 * q[i];
  vh[5] = d0 * py;
  vh[6] = d0 * pz;
  vh[7] = d0 * px;
}

__global__ void k_euler(int N, double dt, const double* __restrict__ V, const double* __restrict__ Om,
                        double* R, double* p) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double px = p[3 * n], py = p[3 * n + 1], pz = p[3 * n + 2];
  const double ox = Om[3 * n], oy = Om[3 * n + 1], oz = Om[3 * n + 2];
  for (int i = 0; i < 3; ++i) R[3 * n + i] += dt * V[3 * n + i];
  double qx = px + dt * (oy * pz - oz * py);
  double qy = py + dt * (oz * px - ox * pz);
  double qz = pz + dt * (ox * py - oy * px);
  const double inv = 1.0 / sqrt(qx * qx + qy * qy + qz * qz);
  p[3 * n] = qx * inv;
  p[3 * n + 1] = qy * inv;
  p[3 * n + 2] = qz * inv;
}

inline unsigned grid1(size_t n, int bs = 256) { return unsigned((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------------
// solver state for one call
// ---------------------------------------------------------------------------------

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

gbi_status setup_call(gbi_ctx* ctx, Setup& s, int N, int trunc, double a, double eta, const double* R) {
  s.N = N;
  s.trunc = trunc;
  s.D = d_of(trunc);
  s.h = s.D - 6;
  s.a = a;
  s.eta = eta;
  const double* sc = scale_tab(trunc);
  const double* sg = self_tab(trunc);
  for (int i = 0; i < 54; ++i) {
    s.scale.v[i] = i < s.D ? sc[i] : 1.0;
    s.selfg.v[i] = i < s.D ? sg[i] : 0.0;
    s.ones.v[i] = 1.0;
    s.minv.v[i] = (i < s.h) ? a / sg[6 + i] : 1.0;
  }
  s.pairs_per_pass = (long long)N * (N - 1);
  GBI_TRY(ensure(ctx, ctx->pos_hi, sizeof(float4) * N));
  GBI_TRY(ensure(ctx, ctx->pos_lo, sizeof(float4) * N));
  GBI_TRY(ensure(ctx, ctx->pos64, sizeof(dpos4) * N));
  k_positions<<<grid1(N), 256, 0, ctx->stream>>>(N, R, P<float4>(ctx->pos_hi), P<float4>(ctx->pos_lo),
                                                 P<dpos4>(ctx->pos64));
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  s.pos = Positions{P<float4>(ctx->pos_hi), P<float4>(ctx->pos_lo), P<dpos4>(ctx->pos64)};
  return GBI_OK;
}

PairArgs pair_args(const Setup& s, const double* x, double* y, double alpha, double beta, int add_self,
                   const Scales& colscale, int col0) {
  PairArgs p;
  p.N = s.N;
  p.a = s.a;
  p.pos = s.pos;
  p.x = x;
  p.x32 = nullptr;
  p.x32lo = nullptr;
  p.wpt = 0;
  p.y = y;
  p.alpha = alpha;
  p.beta = beta;
  p.add_self = add_self;
  for (int i = 0; i < 54; ++i) {
    // colscale is indexed by absolute component; callers pass H-relative scales with col0 = 6
    const int src = i - col0;
    p.colscale[i] = (src >= 0 && src < 54) ? colscale.v[src] : 1.0;
    p.selfg[i] = s.selfg.v[i];
  }
  p.min_r2_bits = nullptr;
  p.x_index = nullptr;
  p.x_stride = 0;
  p.active = nullptr;
  p.sys_of = nullptr;
  p.sys_off = nullptr;
  p.sys_flag = nullptr;
  p.sys_flag_stride = 0;
  return p;
}

// ---------------------------------------------------------------------------------
// Batched GMRES with its control on the device
// ---------------------------------------------------------------------------------
//
// S independent systems (suspensions) share one launch per pass: every vector is
// component-major over all spheres [h][Ntot], sphere n belongs to system sys[n] with
// spheres [off[s], off[s+1]).  Each system has its own Krylov state, Hessenberg
// matrix, Givens rotations, tolerance test and refinement flag; a system that has
// stopped is skipped by every kernel.  A single suspension is the case S = 1.

struct Batch {
  int S = 1;
  int Ntot = 0;
  const int* off = nullptr;   // device [S+1]
  const int* sys = nullptr;   // device [Ntot]
  std::vector<int> h_off;     // host copy of off
};

// Device-resident state of one system's GMRES / refinement.
struct GDev {
  int j;          // Arnoldi index of the vector being expanded
  int active;     // 1 while the current cycle continues
  int iters;      // inner iterations of the current inner solve
  int kdim;       // Krylov dimension reached in the current cycle
  int converged;  // relative residual estimate <= tol
  int breakdown;  // happy breakdown (exact solution in the Krylov space)
  int max_iter, m;
  int enabled;    // refinement: this system still needs a correction
  int pad;
  double bnorm, tol, res, beta, inv_hn;
  double nb;      // |b_s| (reference of the refinement residual)
  double rel;     // |b_s - A q_s| / |b_s|
  double pad2;
};

struct GPtr {     // per-system views into the gstate buffer
  GDev* st;
  double *H, *cs, *sn, *g, *y, *nrm;
  double *h1p, *h2p, *nrmp;   // per-chunk partial sums of the dot products and the norm
  int* nact;                  // systems still active after the current Arnoldi step
  unsigned int* bar;          // grid barrier of the fused single-system step: count, generation, error
  double* fp;                 // its per-block partial sums (two dot-product sets and the norm)
  int S, m, CH;
};

// blocks of the fused single-system Arnoldi step (each holds a slice of the vectors)
constexpr int kFusedBlocks = 64;

// Row chunks per system of the Arnoldi reductions: a few systems get one block per
// component row (so that a single suspension still spreads over many SMs), large
// batches one block per system.
int arnoldi_chunks(int S, int h) { return S >= 64 ? 1 : h; }

size_t gstate_doubles(int m, int S, int CH) {
  return (size_t)S * (sizeof(GDev) / sizeof(double) + 1) + (size_t)S * ((size_t)(m + 1) * m + 5 * (size_t)(m + 1) + 1) +
         (size_t)S * CH * (2 * (size_t)(m + 1) + 1) + (size_t)kFusedBlocks * (2 * (size_t)(m + 1) + 1) + 24;
}

GPtr gptrs(void* base, int m, int S, int CH) {
  GPtr p;
  p.S = S;
  p.m = m;
  p.CH = CH;
  p.st = reinterpret_cast<GDev*>(base);
  double* d = reinterpret_cast<double*>(base) + (size_t)S * (sizeof(GDev) / sizeof(double) + 1);
  p.H = d; d += (size_t)S * (m + 1) * m;
  p.cs = d; d += (size_t)S * (m + 1);
  p.sn = d; d += (size_t)S * (m + 1);
  p.g = d; d += (size_t)S * (m + 1);
  p.y = d; d += (size_t)S * (m + 1);
  p.nrm = d; d += (size_t)S;
  p.h1p = d; d += (size_t)S * (m + 1) * CH;
  p.h2p = d; d += (size_t)S * (m + 1) * CH;
  p.nrmp = d; d += (size_t)S * CH;
  p.nact = reinterpret_cast<int*>(d);
  d += 1;
  p.bar = reinterpret_cast<unsigned int*>(d);
  d += 2;
  p.fp = d;
  return p;
}

__device__ __forceinline__ double block_sum_256(double v) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

// part[(s (m+1) + i) CH + c] = V_i . w over the component rows of chunk c of system s,
// for i <= j_s (block (s, i, c); fixed-order block reduction)
__global__ void bk_dots(const double* __restrict__ V, size_t n, const double* __restrict__ w, int Ntot, int h,
                        const int* __restrict__ off, const GDev* __restrict__ st, int m, int CH, double* part) {
  const int s = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
  const GDev& g = st[s];
  if (!g.active || i > g.j) return;
  const double* v = V + (size_t)i * n;
  const int lo = off[s], hi = off[s + 1];
  const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
  double acc = 0.0;
  for (int q = q0; q < q1; ++q) {
    const size_t b = (size_t)q * Ntot;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) acc += v[b + p] * w[b + p];
  }
  const double t = block_sum_256(acc);
  if (threadIdx.x == 0) part[((size_t)s * (m + 1) + i) * CH + c] = t;
}

// w -= sum_{i <= j_s} coef[s][i] V_i with coef[s][i] = sum over the CH chunk partials (in
// order).  A block whose spheres all belong to one system sums the partials once into
// shared memory; otherwise every thread sums them for its own system.
__global__ void bk_sub(const double* __restrict__ V, size_t n, double* w, int Ntot, const int* __restrict__ sys,
                       const GDev* __restrict__ st, int m, int CH, const double* __restrict__ part) {
  __shared__ double sc[kMaxRestart + 1];
  const int p0 = blockIdx.x * blockDim.x;
  const int pl = min(Ntot - 1, p0 + (int)blockDim.x - 1);
  const int sb = sys[p0];
  const bool uniform = sys[pl] == sb;
  if (uniform) {
    const GDev& g = st[sb];
    if (!g.active) return;
    for (int i = threadIdx.x; i <= g.j; i += blockDim.x) {
      const double* q = part + ((size_t)sb * (m + 1) + i) * CH;
      double acc = 0.0;
      for (int c = 0; c < CH; ++c) acc += q[c];
      sc[i] = acc;
    }
    __syncthreads();
  }
  const int p = p0 + threadIdx.x;
  if (p >= Ntot) return;
  const int s = sys[p];
  const GDev& g = st[s];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  double acc = w[t];
  for (int i = 0; i <= g.j; ++i) {
    double c;
    if (uniform) {
      c = sc[i];
    } else {
      const double* q = part + ((size_t)s * (m + 1) + i) * CH;
      c = 0.0;
      for (int k = 0; k < CH; ++k) c += q[k];
    }
    acc -= c * V[(size_t)i * n + t];
  }
  w[t] = acc;
}

__device__ __forceinline__ bool norm_wanted(const GDev& g, int mode) {
  return !((mode == 0 && !g.active) || (mode == 1 && !g.enabled));
}

// part[s CH + c] = |x_s|^2 over the rows of chunk c (block (s, c)); mode 0: active
// systems, 1: enabled, 2: all
__global__ void bk_norm_part(const double* __restrict__ x, int Ntot, int h, const int* __restrict__ off,
                             const GDev* __restrict__ st, int mode, int CH, double* part) {
  const int s = blockIdx.x, c = blockIdx.y;
  if (!norm_wanted(st[s], mode)) return;
  const int lo = off[s], hi = off[s + 1];
  const int q0 = c * h / CH, q1 = (c + 1) * h / CH;
  double acc = 0.0;
  for (int q = q0; q < q1; ++q) {
    const size_t b = (size_t)q * Ntot;
    for (int p = lo + threadIdx.x; p < hi; p += blockDim.x) acc += x[b + p] * x[b + p];
  }
  const double t = block_sum_256(acc);
  if (threadIdx.x == 0) part[(size_t)s * CH + c] = t;
}

// out[s] = sum of the chunk partials in order
__global__ void bk_norm_sum(const double* __restrict__ part, const GDev* __restrict__ st, int S, int mode, int CH,
                            double* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S || !norm_wanted(st[s], mode)) return;
  double acc = 0.0;
  for (int c = 0; c < CH; ++c) acc += part[(size_t)s * CH + c];
  out[s] = acc;
}

// Hessenberg column j_s, Givens rotations, residual estimate and stopping test of one
// system per block (parallel loads to shared memory, one thread sweeps the rotations).
constexpr int kGmMaxM = 128;
// Hessenberg column j of system s (col[0..j] = the two Gram-Schmidt coefficient sums,
// in shared memory, overwritten), new norm hn: apply the previous rotations, form the
// new one, update g, the residual estimate and the stopping test, store the column.
// Called by one block per system; thread 0 does the serial part.
__device__ void givens_step(const GPtr& p, int s, int j, double hn, double* col, double* scs, double* ssn) {
  GDev* st = p.st + s;
  const int m = p.m;
  const size_t o1 = (size_t)s * (m + 1);
  const int tid = threadIdx.x;
  for (int i = tid; i < j; i += blockDim.x) {
    scs[i] = p.cs[o1 + i];
    ssn[i] = p.sn[o1 + i];
  }
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < j; ++i) {
      const double t1 = col[i], t2 = col[i + 1];
      col[i] = scs[i] * t1 + ssn[i] * t2;
      col[i + 1] = -ssn[i] * t1 + scs[i] * t2;
    }
    col[j + 1] = hn;
    const double hjj = col[j], hj1 = hn;
    const double den = hypot(hjj, hj1);
    const double c = den > 0 ? hjj / den : 1.0, sg = den > 0 ? hj1 / den : 0.0;
    p.cs[o1 + j] = c;
    p.sn[o1 + j] = sg;
    col[j] = den;
    col[j + 1] = 0.0;
    const double gj = p.g[o1 + j];
    p.g[o1 + j + 1] = -sg * gj;
    p.g[o1 + j] = c * gj;
    st->iters += 1;
    st->kdim = j + 1;
    st->res = fabs(p.g[o1 + j + 1]) / st->bnorm;
    st->converged = st->res <= st->tol;
    st->breakdown = hn <= 1e-300;
    const bool stop = st->converged || st->breakdown || st->iters >= st->max_iter || j + 1 >= m;
    if (stop) {
      st->active = 0;
    } else {
      st->inv_hn = 1.0 / hn;
      st->j = j + 1;
      atomicAdd(p.nact, 1);
    }
  }
  __syncthreads();
  double* H = p.H + (size_t)s * (m + 1) * m;
  for (int i = tid; i <= j + 1; i += blockDim.x) H[(size_t)i * m + j] = col[i];
}

__global__ void bk_finalize(GPtr p) {
  const int s = blockIdx.x;
  GDev* st = p.st + s;
  if (!st->active) return;
  __shared__ double col[kGmMaxM + 1], scs[kGmMaxM], ssn[kGmMaxM];
  const int j = st->j, m = p.m;
  const size_t o1 = (size_t)s * (m + 1);
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double* a1 = p.h1p + (o1 + i) * p.CH;
    const double* a2 = p.h2p + (o1 + i) * p.CH;
    double c1 = 0.0, c2 = 0.0;
    for (int c = 0; c < p.CH; ++c) {
      c1 += a1[c];
      c2 += a2[c];
    }
    col[i] = c1 + c2;
  }
  __shared__ double s_hn;
  if (threadIdx.x == 0) {
    double nrm = 0.0;
    for (int c = 0; c < p.CH; ++c) nrm += p.nrmp[(size_t)s * p.CH + c];
    s_hn = sqrt(fmax(0.0, nrm));
  }
  __syncthreads();
  givens_step(p, s, j, s_hn, col, scs, ssn);
}

// Arnoldi source of the next pair pass, written by the kernels that produce V_j:
// FP32 records (PairArgs::x32, ncp floats per sphere, zero padding) or FP64
// component-major, both scaled by the column multipliers minv.
struct SrcOut {
  float* rec;
  double* dbl;
  int ncp;
  Scales minv;
};

__device__ __forceinline__ void write_src(const SrcOut& o, int Ntot, int h, int q, int p, double v) {
  if (o.rec != nullptr) {
    float* r = o.rec + (size_t)p * o.ncp;
    r[q] = float(v * o.minv.v[q]);
    if (q == 0)
      for (int k = h; k < o.ncp; ++k) r[k] = 0.f;
  } else if (o.dbl != nullptr) {
    o.dbl[(size_t)q * Ntot + p] = v * o.minv.v[q];
  }
}

// V_{j_s} = w / h for the newly advanced j_s (and its Arnoldi source)
__global__ void bk_scale(double* V, size_t n, const double* __restrict__ w, int Ntot, const int* __restrict__ sys,
                         const GDev* __restrict__ st, SrcOut src) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  const GDev& g = st[sys[p]];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  const double v = w[t] * g.inv_hn;
  V[(size_t)g.j * n + t] = v;
  write_src(src, Ntot, gridDim.y, blockIdx.y, p, v);
}

// ---------------------------------------------------------------------------------
// Fused Arnoldi step of a single system: both Gram-Schmidt rounds, the norm, the
// Givens update and V_{j+1} (with its pair-pass source) in one kernel of kFusedBlocks
// blocks, each owning a contiguous slice of the vectors, separated by three grid-wide
// barriers.  Partial sums are combined in block order by every block (identical
// results everywhere), so the result does not depend on timing.  The blocks must be
// co-resident: 64 blocks of 256 threads on a 152-SM GPU that runs nothing else in the
// stream meanwhile.  Each barrier wait is bounded; a block that gives up records an
// error (bar[2]) and returns, and the host reports GBI_ERR_TIMEOUT.
// ---------------------------------------------------------------------------------

constexpr long long kBarrierLimit = 1ll << 22;   // polling rounds (with back-off) per barrier

__device__ bool grid_barrier(unsigned int* bar, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = atomicAdd(&bar[1], 0u);   // generation before arriving
    __threadfence();
    int ok = 1;
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long it = 0;
      while (atomicAdd(&bar[1], 0u) == g) {
        if (++it > kBarrierLimit) {
          atomicExch(&bar[2], 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// sum over the block in a fixed order; the leading barrier makes back-to-back calls safe
__device__ __forceinline__ double block_sum_ordered(double v, double* sh) {
  __syncthreads();
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  return sh[0];
}

// part[i G + b] = V_i . w over [t0, t1) for i <= j: warp k of the block takes
// i = k, k + nwarps, ...; lanes stride the slice and a shuffle tree sums them (fixed order)
__device__ __forceinline__ void slice_dots(const double* __restrict__ V, size_t n, const double* __restrict__ w,
                                           int j, size_t t0, size_t t1, double* part, int G, int b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i <= j; i += nw) {
    const double* v = V + (size_t)i * n;
    double acc = 0.0;
    for (size_t t = t0 + lane; t < t1; t += 32) acc += v[t] * w[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[(size_t)i * G + b] = acc;
  }
}

__global__ void __launch_bounds__(256) bk_step_fused(double* V, size_t n, double* w, int Ntot, int h, GPtr p,
                                                     SrcOut so) {
  __shared__ double sh[256];
  __shared__ double c1[kGmMaxM + 1], c2[kGmMaxM + 1], scs[kGmMaxM], ssn[kGmMaxM];
  __shared__ double s_hn;
  __shared__ int s_ok;
  const GDev* st = p.st;
  if (!st->active) return;   // the same decision in every block: nothing writes the state yet
  const int j = st->j, m = p.m;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const size_t L = (n + G - 1) / G;
  const size_t t0 = (size_t)b * L, t1 = min(n, t0 + L);
  double* part1 = p.fp;
  double* part2 = p.fp + (size_t)(m + 1) * G;
  double* partn = p.fp + 2 * (size_t)(m + 1) * G;
  // (A) partial V_i . w: warp w of the block takes i = w, w + 8, ... (no block barrier)
  slice_dots(V, n, w, j, t0, t1, part1, G, b);
  if (!grid_barrier(p.bar, &s_ok)) return;
  // (B) w1 = w - sum c1_i V_i on the slice, then partial V_i . w1
  for (int i = tid; i <= j; i += blockDim.x) {
    double c = 0.0;
    for (int q = 0; q < G; ++q) c += part1[(size_t)i * G + q];
    c1[i] = c;
  }
  __syncthreads();
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    double a = w[t];
    for (int i = 0; i <= j; ++i) a -= c1[i] * V[(size_t)i * n + t];
    w[t] = a;
  }
  __syncthreads();
  slice_dots(V, n, w, j, t0, t1, part2, G, b);
  if (!grid_barrier(p.bar, &s_ok)) return;
  // (C) w2 = w1 - sum c2_i V_i, partial |w2|^2
  for (int i = tid; i <= j; i += blockDim.x) {
    double c = 0.0;
    for (int q = 0; q < G; ++q) c += part2[(size_t)i * G + q];
    c2[i] = c;
  }
  __syncthreads();
  double nacc = 0.0;
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    double a = w[t];
    for (int i = 0; i <= j; ++i) a -= c2[i] * V[(size_t)i * n + t];
    w[t] = a;
    nacc += a * a;
  }
  nacc = block_sum_ordered(nacc, sh);
  if (tid == 0) partn[b] = nacc;
  if (!grid_barrier(p.bar, &s_ok)) return;
  // (D) h_{j+1,j} = |w2|, V_{j+1} = w2 / h and its source; block 0 updates the rotations
  if (tid == 0) {
    double nrm = 0.0;
    for (int q = 0; q < G; ++q) nrm += partn[q];
    s_hn = sqrt(fmax(0.0, nrm));
  }
  __syncthreads();
  const double hn = s_hn;
  const double inv = hn > 1e-300 ? 1.0 / hn : 0.0;
  for (size_t t = t0 + tid; t < t1; t += blockDim.x) {
    const double v = w[t] * inv;
    V[(size_t)(j + 1) * n + t] = v;
    const int q = int(t / (size_t)Ntot);
    write_src(so, Ntot, h, q, int(t - (size_t)q * Ntot), v);
  }
  if (b == 0) {
    for (int i = tid; i <= j; i += blockDim.x) c1[i] += c2[i];
    __syncthreads();
    givens_step(p, 0, j, hn, c1, scs, ssn);
  }
}

// End of one device-looped Arnoldi step: keep looping while any system is still active
// (the WHILE node of the cycle graph reads the value set here), and reset the count.
__global__ void bk_continue(GPtr p, cudaGraphConditionalHandle h) {
  const int v = *p.nact;
  *p.nact = 0;
  cudaGraphSetConditional(h, v > 0 ? 1u : 0u);
}

// start of a GMRES cycle for every enabled system: beta = |V_0|, g = (beta, 0, ...)
__global__ void bk_init_cycle(GPtr p, int first) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *p.nact = 0;
  if (s >= p.S) return;
  GDev* st = p.st + s;
  const int m = p.m;
  if (first) st->iters = 0;
  st->j = 0;
  st->kdim = 0;
  st->breakdown = 0;
  if (!st->enabled || (!first && st->converged)) {
    st->active = 0;
    return;
  }
  const double beta = sqrt(fmax(0.0, p.nrm[s]));
  if (first) st->bnorm = beta;
  st->beta = beta;
  double* g = p.g + (size_t)s * (m + 1);
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  st->res = st->bnorm > 0 ? beta / st->bnorm : 0.0;
  st->converged = st->res <= st->tol;
  st->active = (!st->converged && st->iters < st->max_iter && beta > 0) ? 1 : 0;
  st->inv_hn = beta > 0 ? 1.0 / beta : 0.0;
}

__global__ void bk_scale0(double* V0, int Ntot, const int* __restrict__ sys, const GDev* __restrict__ st,
                          SrcOut src) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  const GDev& g = st[sys[p]];
  if (!g.active) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  const double v = V0[t] * g.inv_hn;
  V0[t] = v;
  write_src(src, Ntot, gridDim.y, blockIdx.y, p, v);
}

// y_s = H_s^-1 g_s on the kdim leading rows (column-oriented back substitution)
__global__ void bk_solve_y(GPtr p) {
  const int s = blockIdx.x;
  const GDev* st = p.st + s;
  const int k = st->kdim, m = p.m;
  if (k == 0) return;
  const double* H = p.H + (size_t)s * (m + 1) * m;
  const size_t o1 = (size_t)s * (m + 1);
  __shared__ double rhs[kGmMaxM], yv[kGmMaxM];
  for (int i = threadIdx.x; i < k; i += blockDim.x) rhs[i] = p.g[o1 + i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) yv[i] = rhs[i] / H[(size_t)i * m + i];
    __syncthreads();
    for (int r = threadIdx.x; r < i; r += blockDim.x) rhs[r] -= H[(size_t)r * m + i] * yv[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) p.y[o1 + i] = yv[i];
}

// u += minv * sum_{i < kdim_s} y_s[i] V_i  (systems whose cycle ran)
__global__ void bk_update(const double* __restrict__ V, size_t n, int Ntot, const int* __restrict__ sys, GPtr p,
                          Scales minv, double* u) {
  const int pp = blockIdx.x * blockDim.x + threadIdx.x;
  if (pp >= Ntot) return;
  const int s = sys[pp];
  const int k = p.st[s].kdim;
  if (k == 0) return;
  const size_t t = (size_t)blockIdx.y * Ntot + pp;
  const double* y = p.y + (size_t)s * (p.m + 1);
  double acc = 0.0;
  for (int i = 0; i < k; ++i) acc += y[i] * V[(size_t)i * n + t];
  u[t] += minv.v[blockIdx.y] * acc;
}

// refinement bookkeeping: mode 0 stores |b_s| (from nrm), mode 1 sets rel and enabled
__global__ void bk_refine(GPtr p, int mode, double rtol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.S) return;
  GDev* st = p.st + s;
  const double v = sqrt(fmax(0.0, p.nrm[s]));
  if (mode == 0) {
    st->nb = v;
    st->enabled = v > 0 ? 1 : 0;
    st->rel = v > 0 ? 1.0 : 0.0;
  } else if (st->enabled) {
    st->rel = st->nb > 0 ? v / st->nb : 0.0;
    st->enabled = st->rel > rtol ? 1 : 0;
  }
}

// x += d on enabled systems
__global__ void bk_axpy_enabled(const double* __restrict__ d, int Ntot, const int* __restrict__ sys,
                                const GDev* __restrict__ st, double* x) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= Ntot) return;
  if (!st[sys[p]].enabled) return;
  const size_t t = (size_t)blockIdx.y * Ntot + p;
  x[t] += d[t];
}

// Restarted right-preconditioned GMRES(m) on every active system of the batch for
// G^HH u = rhs (internal coordinates).  u holds the initial guess (zero or warm).
// Arnoldi (classical Gram-Schmidt twice), Givens rotations, the stopping tests and
// the triangular solves run on the device in FP64; the host launches the iterations
// in chunks (replayed from a CUDA graph when the stream allows capture) and reads the
// systems' small states once per chunk.
gbi_status gmres_batch(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const double* rhs, double* u,
                       bool u_is_zero, double tol, int restart, int max_iter, gbi_info* info, int& iters,
                       double& relres, std::vector<GDev>& hst, double outer_rtol = 0.0);

// Where the kernels producing V_j put the next pair pass's source (see SrcOut).
SrcOut src_out(const Setup& s, int precision, void* xsrc) {
  SrcOut o;
  o.rec = precision == 1 ? static_cast<float*>(xsrc) : nullptr;
  o.dbl = precision == 1 ? nullptr : static_cast<double*>(xsrc);
  o.ncp = (s.h + 3) & ~3;
  o.minv = s.minv;
  return o;
}

// kChunk Arnoldi iterations of every active system: pair pass on the source of V_j
// (written by the previous bk_scale / bk_scale0), two rounds of classical Gram-Schmidt,
// norm, Givens update and V_{j+1} with its source -- eight kernels per iteration.  With
// fused set and a single system the seven kernels after the pair pass are replaced by
// bk_step_fused; that is faster for direct launches, while inside the cycle graph the
// separate kernels (graph launch overhead about a microsecond each) measured faster than
// the fused kernel's three grid barriers.
gbi_status launch_chunk(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const GPtr& gp, int m,
                        double* Vb, double* w, void* xsrc, int kChunk, bool fused) {
  const int S = B.S, Ntot = B.Ntot, h = s.h;
  const size_t n = (size_t)Ntot * h;
  const dim3 g2((Ntot + 255) / 256, h);
  PairArgs pa = pair_args(s, precision == 1 ? nullptr : static_cast<const double*>(xsrc), w, 1.0, 0.0, 1, s.ones,
                          6);
  if (precision == 1) pa.x32 = static_cast<const float*>(xsrc);
  pa.sys_of = B.sys;
  pa.sys_off = B.off;
  pa.sys_flag = &gp.st[0].active;
  pa.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
  const SrcOut so = src_out(s, precision, xsrc);
  const dim3 gd(S, m + 1, gp.CH);
  for (int c = 0; c < kChunk; ++c) {
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, precision, pa));
    if (fused && S == 1) {
      // a single system launched step by step: the whole orthogonalisation in one kernel
      bk_step_fused<<<kFusedBlocks, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, gp, so);
      ++ctx->launches;
      continue;
    }
    bk_dots<<<gd, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp.st, m, gp.CH, gp.h1p);
    bk_sub<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, m, gp.CH, gp.h1p);
    bk_dots<<<gd, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, h, B.off, gp.st, m, gp.CH, gp.h2p);
    bk_sub<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, m, gp.CH, gp.h2p);
    bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(w, Ntot, h, B.off, gp.st, 0, gp.CH, gp.nrmp);
    bk_finalize<<<S, 128, 0, ctx->stream>>>(gp);
    bk_scale<<<g2, 256, 0, ctx->stream>>>(Vb, n, w, Ntot, B.sys, gp.st, so);
    ctx->launches += 7;
  }
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

// Per-system GMRES set-up.  With outer_rtol > 0 (an inner solve of the refinement) the
// tolerance relative to the current residual r is loosened to 0.1 outer_rtol |b| / |r|
// when that is larger than tol: the solve only has to bring |r| a decade below the
// target, so a refinement sweep that starts close to it needs few iterations.
__global__ void bk_setup(GPtr p, double tol, int max_iter, double outer_rtol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.S) return;
  GDev* st = p.st + s;
  if (s == 0) {
    p.bar[0] = 0u;   // arrivals
    p.bar[2] = 0u;   // error flag
  }
  st->tol = outer_rtol > 0 ? fmax(tol, 0.1 * outer_rtol / fmax(st->rel, 1e-300)) : tol;
  st->max_iter = max_iter;
  st->m = p.m;
  st->active = 0;
  st->converged = 0;
  st->iters = 0;
}

gbi_status gmres_batch(gbi_ctx* ctx, const Setup& s, const Batch& B, int precision, const double* rhs, double* u,
                       bool u_is_zero, double tol, int restart, int max_iter, gbi_info* info, int& iters,
                       double& relres, std::vector<GDev>& hst, double outer_rtol) {
  constexpr int kChunk = 6;
  const int S = B.S, Ntot = B.Ntot, h = s.h;
  const size_t n = (size_t)Ntot * h;
  const int m = std::max(1, std::min(restart, kMaxRestart));
  GBI_TRY(ensure(ctx, ctx->krylov, sizeof(double) * n * (m + 1)));
  GBI_TRY(ensure(ctx, ctx->w, sizeof(double) * n));
  GBI_TRY(ensure(ctx, ctx->gstate, sizeof(double) * gstate_doubles(m, S, arnoldi_chunks(S, h))));
  // gathered Arnoldi source: FP64 component-major, or FP32 records of round4(h) floats
  GBI_TRY(ensure(ctx, ctx->x32, std::max(sizeof(double) * n, sizeof(float) * (size_t)Ntot * ((h + 3) & ~3))));
  double* Vb = P<double>(ctx->krylov);
  double* w = P<double>(ctx->w);
  void* xsrc = ctx->x32.p;
  const GPtr gp = gptrs(ctx->gstate.p, m, S, arnoldi_chunks(S, h));
  const dim3 g2((Ntot + 255) / 256, h);
  const int sblk = (S + 127) / 128;
  iters = 0;
  relres = 0.0;
  bk_setup<<<sblk, 128, 0, ctx->stream>>>(gp, tol, std::max(0, max_iter), outer_rtol);
  ++ctx->launches;
  // cycle graph: a WHILE node whose body is one Arnoldi step of every active system
  // followed by bk_continue; the loop runs on the device until no system is active, so a
  // GMRES cycle costs one graph launch and one read of the per-system states.  Built
  // once per buffer set and replayed afterwards.
  const bool graphs = ctx->allow_graphs && ctx->stream != nullptr && !ctx->prof;
  if (graphs) {
    const void* key[8] = {Vb, w, xsrc, ctx->gstate.p, B.sys, B.off, s.pos.hi, s.pos.p64};
    const long long ikey[6] = {(long long)n, S, m, precision, s.trunc, Ntot};
    bool same = ctx->chunk_exec != nullptr;
    for (int i = 0; i < 8 && same; ++i) same = ctx->chunk_key[i] == key[i];
    for (int i = 0; i < 6 && same; ++i) same = ctx->chunk_ikey[i] == ikey[i];
    if (!same) {
      if (ctx->chunk_exec) cudaGraphExecDestroy(ctx->chunk_exec);
      ctx->chunk_exec = nullptr;
      cudaGraph_t graph = nullptr;
      GBI_CHECK(cudaGraphCreate(&graph, 0));
      cudaGraphConditionalHandle handle;
      cudaError_t e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
      const long long saved = ctx->launches;
      gbi_status st = GBI_OK;
      if (e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(ctx->stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          st = launch_chunk(ctx, s, B, precision, gp, m, Vb, w, xsrc, 1, false);
          bk_continue<<<1, 1, 0, ctx->stream>>>(gp, handle);
          ++ctx->launches;
          cudaGraph_t body = nullptr;
          const cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &body);
          if (e == cudaSuccess) e = e2;
        }
      }
      ctx->chunk_nodes = int(ctx->launches - saved);   // kernels per loop iteration
      ctx->launches = saved;
      if (st == GBI_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ctx->chunk_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (st != GBI_OK) return st;
      GBI_CHECK(e);
      for (int i = 0; i < 8; ++i) ctx->chunk_key[i] = key[i];
      for (int i = 0; i < 6; ++i) ctx->chunk_ikey[i] = ikey[i];
    }
  }
  hst.resize(S);
  bool first = true;
  std::vector<int> before(S, 0);
  while (true) {
    // V_0 = rhs - A u on the enabled systems, beta_s = |V_0,s|
    GBI_CHECK(cudaMemcpyAsync(Vb, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (!(first && u_is_zero)) {
      PairArgs pr = pair_args(s, u, Vb, -1.0, 1.0, 1, s.ones, 6);
      pr.sys_of = B.sys;
      pr.sys_off = B.off;
      pr.sys_flag = &gp.st[0].enabled;
      pr.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
      GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, precision, pr));
      if (info) {
        (precision == 1 ? info->matvecs_f32 : info->matvecs_f64) += 1;
        for (int q = 0; q < S; ++q)
          if (hst[q].enabled) info->pair_interactions += (long long)(B.h_off[q + 1] - B.h_off[q]) * (B.h_off[q + 1] - B.h_off[q] - 1);
      }
    }
    bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(Vb, Ntot, h, B.off, gp.st, 1, gp.CH, gp.nrmp);
    bk_norm_sum<<<(S + 127) / 128, 128, 0, ctx->stream>>>(gp.nrmp, gp.st, S, 1, gp.CH, gp.nrm);
    bk_init_cycle<<<sblk, 128, 0, ctx->stream>>>(gp, first ? 1 : 0);
    bk_scale0<<<g2, 256, 0, ctx->stream>>>(Vb, Ntot, B.sys, gp.st, src_out(s, precision, xsrc));
    ctx->launches += 4;
    GBI_CHECK(cudaGetLastError());
    if (first)
      for (int q = 0; q < S; ++q) before[q] = 0;      // bk_init_cycle restarts the counters
    else
      for (int q = 0; q < S; ++q) before[q] = hst[q].iters;
    first = false;
    auto account = [&](int nsteps) {
      // states after the launched steps: pair work of the systems that took them
      int live = 0;
      for (int q = 0; q < S; ++q) {
        const int d = hst[q].iters - before[q];
        before[q] = hst[q].iters;
        live = std::max(live, d);
        if (info) info->pair_interactions += (long long)d * (B.h_off[q + 1] - B.h_off[q]) * (B.h_off[q + 1] - B.h_off[q] - 1);
      }
      if (info) (precision == 1 ? info->matvecs_f32 : info->matvecs_f64) += live;
      ctx->stat_dead[precision * 9 + SET_H * 3 + SET_H] += std::max(0, nsteps - live);
      return live;
    };
    auto read_states = [&]() -> gbi_status {
      ctx->hbatch.resize(sizeof(GDev) * S + sizeof(unsigned int) * 3);
      GBI_CHECK(cudaMemcpyAsync(ctx->hbatch.data(), gp.st, sizeof(GDev) * S, cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaMemcpyAsync(ctx->hbatch.data() + sizeof(GDev) * S, gp.bar, sizeof(unsigned int) * 3,
                                cudaMemcpyDeviceToHost, ctx->stream));
      GBI_CHECK(cudaStreamSynchronize(ctx->stream));
      std::memcpy(hst.data(), ctx->hbatch.data(), sizeof(GDev) * S);
      unsigned int bar[3];
      std::memcpy(bar, ctx->hbatch.data() + sizeof(GDev) * S, sizeof(bar));
      if (bar[2] != 0u) {
        ctx->err = "fused Arnoldi step: a grid barrier wait gave up";
        return GBI_ERR_TIMEOUT;
      }
      return GBI_OK;
    };
    if (graphs) {
      // the whole cycle's Arnoldi steps in one launch; the loop ran max(1, most steps) times
      GBI_CHECK(cudaGraphLaunch(ctx->chunk_exec, ctx->stream));
      GBI_TRY(read_states());
      int most = 0;
      for (int q = 0; q < S; ++q) most = std::max(most, hst[q].iters - before[q]);
      const int steps = std::max(1, most);
      ctx->launches += (long long)steps * ctx->chunk_nodes;
      account(steps);
    } else {
      // host-driven: chunks of kChunk steps with a state read after each
      GBI_TRY(read_states());
      bool any = false;
      for (int q = 0; q < S; ++q) any = any || hst[q].active;
      while (any) {
        GBI_TRY(launch_chunk(ctx, s, B, precision, gp, m, Vb, w, xsrc, kChunk, true));
        GBI_TRY(read_states());
        account(kChunk);
        any = false;
        for (int q = 0; q < S; ++q) any = any || hst[q].active;
      }
    }
    bk_solve_y<<<S, 128, 0, ctx->stream>>>(gp);
    bk_update<<<g2, 256, 0, ctx->stream>>>(Vb, n, Ntot, B.sys, gp, s.minv, u);
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    bool restart_any = false;
    for (int q = 0; q < S; ++q) {
      const GDev& g = hst[q];
      iters = std::max(iters, g.iters);
      if (g.enabled && g.kdim > 0 && !g.converged && !g.breakdown && g.iters < g.max_iter) restart_any = true;
    }
    if (!restart_any) break;
  }
  relres = 0.0;
  for (int q = 0; q < S; ++q)
    if (hst[q].enabled) relres = std::max(relres, hst[q].res);
  return GBI_OK;
}

bool valid_params(const gbi_params* p) {
  if (!p) return false;
  if (!(p->a > 0) || !(p->eta > 0)) return false;
  if (p->trunc < 2 || p->trunc > 4) return false;
  if (p->precision < 0 || p->precision > 3) return false;
  return true;
}

// The full solve for a batch of independent suspensions (S = 1: one suspension).
// Inputs and outputs are concatenated over the systems ([Ntot][3], [Ntot][h]).
gbi_status solve_core(gbi_ctx* ctx, const gbi_params* prm, const Batch& B, const double* R, const double* Va,
                      const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                      double* Omega, double* QH, int warm_start, gbi_info* inf) {
  const int N = B.Ntot, S = B.S;
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, prm->trunc, prm->a, prm->eta, R));
  long long pairs_all = 0;
  for (int q = 0; q < S; ++q) {
    const long long ns = B.h_off[q + 1] - B.h_off[q];
    pairs_all += ns * (ns - 1);
  }
  s.pairs_per_pass = pairs_all;
  const int D = s.D, h = s.h;
  const size_t nh = (size_t)N * h;
  const dim3 g2((N + 255) / 256, h);
  const int sblk = (S + 127) / 128;
  // arithmetic of the refinement residual (FP64, or double-float for precision 2 and 3)
  // and of the right-hand-side and output passes (the same, or FP32 for precision 3)
  const int hp = prm->precision >= 2 ? 2 : 0;
  const int io = prm->precision == 3 ? 1 : hp;
  const int restart = std::max(1, std::min(prm->restart > 0 ? prm->restart : 40, kMaxRestart));
  GBI_TRY(ensure(ctx, ctx->xQ, sizeof(double) * (size_t)N * D));
  GBI_TRY(ensure(ctx, ctx->xVH, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->b, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->r, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->delta, sizeof(double) * nh));
  GBI_TRY(ensure(ctx, ctx->xVL, sizeof(double) * 6 * N));
  GBI_TRY(ensure(ctx, ctx->minr2, sizeof(unsigned int)));
  GBI_TRY(ensure(ctx, ctx->gstate, sizeof(double) * gstate_doubles(restart, S, arnoldi_chunks(S, h))));
  double* xF = P<double>(ctx->xQ);              // rows 0..5 of the full vector
  double* xQH = P<double>(ctx->xQ) + (size_t)6 * N;
  double* b = P<double>(ctx->b);
  double* r = P<double>(ctx->r);
  double* dl = P<double>(ctx->delta);
  const GPtr gp = gptrs(ctx->gstate.p, restart, S, arnoldi_chunks(S, h));
  const double c2a = s.scale.v[3];
  Scales hscale;
  for (int i = 0; i < 54; ++i) hscale.v[i] = (i < h) ? s.scale.v[6 + i] : 1.0;
  auto batched = [&](PairArgs p, const int* flag) {
    p.sys_of = B.sys;
    p.sys_off = B.off;
    p.sys_flag = flag;
    p.sys_flag_stride = int(sizeof(GDev) / sizeof(int));
    return p;
  };
  std::vector<GDev> hst(S);

  // inputs -> internal coordinates
  k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, c2a, Fe, Te, xF);
  // b = -8 pi eta V^H
  k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, hscale, -8.0 * kPi * s.eta, b);
  ctx->launches += 2;
  GBI_CHECK(cudaGetLastError());
  // b -= G^HL F^L, with the overlap scan
  const unsigned int init_bits = 0x7f7fffffu;
  GBI_CHECK(cudaMemcpyAsync(ctx->minr2.p, &init_bits, sizeof(unsigned int), cudaMemcpyHostToDevice, ctx->stream));
  {
    PairArgs p = batched(pair_args(s, xF, b, -1.0, 1.0, 0, s.ones, 0), nullptr);
    p.min_r2_bits = P<unsigned int>(ctx->minr2);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_L, io, p));
    (io == 1 ? inf->matvecs_f32 : inf->matvecs_f64) += 1;
    inf->pair_interactions += pairs_all;
  }
  if (prm->min_sep > 0) {
    unsigned int bits = 0;
    GBI_CHECK(cudaMemcpyAsync(&bits, ctx->minr2.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    float mr2;
    std::memcpy(&mr2, &bits, sizeof(float));
    inf->min_separation = pairs_all > 0 ? std::sqrt(double(mr2)) / s.a : 0.0;
    if (pairs_all > 0 && inf->min_separation < prm->min_sep) return GBI_ERR_OVERLAP;
  }

  // initial guess
  bool zero = true;
  if (warm_start) {
    k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, QH, hscale, 1.0, xQH);
    ++ctx->launches;
    zero = false;
  } else {
    GBI_CHECK(cudaMemsetAsync(xQH, 0, sizeof(double) * nh, ctx->stream));
  }
  const int max_iter = prm->max_iter > 0 ? prm->max_iter : 1000;
  const double rtol = prm->rtol > 0 ? prm->rtol : 1e-10;
  // |b_s| per system
  bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(b, N, h, B.off, gp.st, 2, gp.CH, gp.nrmp);
  bk_norm_sum<<<(S + 127) / 128, 128, 0, ctx->stream>>>(gp.nrmp, gp.st, S, 2, gp.CH, gp.nrm);
  bk_refine<<<sblk, 128, 0, ctx->stream>>>(gp, 0, rtol);
  ctx->launches += 3;
  auto read_state = [&]() -> gbi_status {
    ctx->hbatch.resize(sizeof(GDev) * S);
    GBI_CHECK(cudaMemcpyAsync(ctx->hbatch.data(), gp.st, sizeof(GDev) * S, cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(hst.data(), ctx->hbatch.data(), sizeof(GDev) * S);
    return GBI_OK;
  };
  auto pairs_enabled = [&]() {
    long long c = 0;
    for (int q = 0; q < S; ++q)
      if (hst[q].enabled) {
        const long long ns = B.h_off[q + 1] - B.h_off[q];
        c += ns * (ns - 1);
      }
    return c;
  };
  GBI_TRY(read_state());
  bool converged = false;
  if (prm->precision == 0) {
    int it = 0;
    double rr = 0.0;
    GBI_TRY(gmres_batch(ctx, s, B, 0, b, xQH, zero, rtol, restart, max_iter, inf, it, rr, hst));
    inf->iters += it;
    // true FP64 residual per system
    GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
    PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, 0, p));
    inf->matvecs_f64 += 1;
    inf->pair_interactions += pairs_enabled();
    bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(r, N, h, B.off, gp.st, 1, gp.CH, gp.nrmp);
    bk_norm_sum<<<(S + 127) / 128, 128, 0, ctx->stream>>>(gp.nrmp, gp.st, S, 1, gp.CH, gp.nrm);
    bk_refine<<<sblk, 128, 0, ctx->stream>>>(gp, 1, rtol);
    ctx->launches += 3;
    GBI_TRY(read_state());
  } else {
    // mixed precision: r = b - A_hp x; A_32 d = r (FP32 pair sums, FP64 Arnoldi); x += d
    const double inner = prm->inner_rtol > 0 ? prm->inner_rtol : 1e-5;
    const int max_refine = prm->max_refine > 0 ? prm->max_refine : 8;
    for (int sweep = 0;; ++sweep) {
      GBI_CHECK(cudaMemcpyAsync(r, b, sizeof(double) * nh, cudaMemcpyDeviceToDevice, ctx->stream));
      if (!(zero && sweep == 0)) {
        PairArgs p = batched(pair_args(s, xQH, r, -1.0, 1.0, 1, s.ones, 6), &gp.st[0].enabled);
        GBI_CHECK(run_pairs(ctx, s.trunc, SET_H, SET_H, hp, p));
        inf->matvecs_f64 += 1;
        inf->pair_interactions += pairs_enabled();
        bk_norm_part<<<dim3(S, gp.CH), 256, 0, ctx->stream>>>(r, N, h, B.off, gp.st, 1, gp.CH, gp.nrmp);
        bk_norm_sum<<<(S + 127) / 128, 128, 0, ctx->stream>>>(gp.nrmp, gp.st, S, 1, gp.CH, gp.nrm);
        bk_refine<<<sblk, 128, 0, ctx->stream>>>(gp, 1, rtol);
        ctx->launches += 3;
      }
      if (sweep > 0) inf->refinements += 1;
      if (sweep >= max_refine || inf->iters >= max_iter) {
        GBI_TRY(read_state());
        break;
      }
      int it = 0;
      double rr = 0.0;
      GBI_CHECK(cudaMemsetAsync(dl, 0, sizeof(double) * nh, ctx->stream));
      GBI_TRY(gmres_batch(ctx, s, B, 1, r, dl, true, inner, restart, max_iter - inf->iters, inf, it, rr, hst,
                          rtol));
      inf->iters += it;
      bool any = false;
      for (int q = 0; q < S; ++q) any = any || hst[q].enabled;
      if (!any) break;       // every system met the tolerance at this sweep's residual
      bk_axpy_enabled<<<g2, 256, 0, ctx->stream>>>(dl, N, B.sys, gp.st, xQH);
      ++ctx->launches;
      GBI_CHECK(cudaGetLastError());
    }
  }
  converged = true;
  inf->rel_residual = 0.0;
  for (int q = 0; q < S; ++q) {
    inf->rel_residual = std::max(inf->rel_residual, hst[q].rel);
    if (hst[q].rel > rtol) converged = false;
  }
  // outputs: 8 pi eta x^{V,L} = -(G^LL F^L + G^LH Q^H) incl. self
  {
    PairArgs p = batched(pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1,
                                   s.ones, 0),
                         nullptr);
    GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, io, p));
    (io == 1 ? inf->matvecs_f32 : inf->matvecs_f64) += 1;
    inf->pair_interactions += pairs_all;
  }
  k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, c2a, P<double>(ctx->xVL), Va, Oa, V, Omega);
  ++ctx->launches;
  if (QH) {
    k_unpack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, xQH, hscale, QH);
    ++ctx->launches;
  }
  GBI_CHECK(cudaGetLastError());
  if (prm->min_sep <= 0) {
    unsigned int bits = 0;
    GBI_CHECK(cudaMemcpyAsync(&bits, ctx->minr2.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    float mr2;
    std::memcpy(&mr2, &bits, sizeof(float));
    inf->min_separation = pairs_all > 0 ? std::sqrt(double(mr2)) / s.a : 0.0;
  } else {
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  }
  return converged ? GBI_OK : GBI_ERR_NOT_CONVERGED;
}

// S = 1 batch over the spheres [0, N): offsets and system ids in the context workspace
gbi_status single_batch(gbi_ctx* ctx, int N, Batch& B) {
  GBI_TRY(ensure(ctx, ctx->boff, sizeof(int) * 2));
  GBI_TRY(ensure(ctx, ctx->bsys, sizeof(int) * (size_t)std::max(N, 1)));
  const int off[2] = {0, N};
  GBI_CHECK(cudaMemcpyAsync(ctx->boff.p, off, sizeof(off), cudaMemcpyHostToDevice, ctx->stream));
  GBI_CHECK(cudaMemsetAsync(ctx->bsys.p, 0, sizeof(int) * (size_t)N, ctx->stream));
  B.S = 1;
  B.Ntot = N;
  B.off = P<int>(ctx->boff);
  B.sys = P<int>(ctx->bsys);
  B.h_off.assign({0, N});
  return GBI_OK;
}

__global__ void k_fill_sys(int S, const int* __restrict__ off, int* sys) {
  const int s = blockIdx.x;
  for (int p = off[s] + threadIdx.x; p < off[s + 1]; p += blockDim.x) sys[p] = s;
}

bool valid_offsets(int nsys, const int* off) {
  if (off[0] != 0) return false;
  for (int q = 0; q < nsys; ++q)
    if (off[q + 1] < off[q]) return false;
  return true;
}

// Device copies of a batch layout (system offsets and the system of every sphere).
gbi_status make_batch(gbi_ctx* ctx, int nsys, const int* offsets_host, Batch& B) {
  const int N = offsets_host[nsys];
  GBI_TRY(ensure(ctx, ctx->boff, sizeof(int) * (size_t)(nsys + 1)));
  GBI_TRY(ensure(ctx, ctx->bsys, sizeof(int) * (size_t)N));
  GBI_CHECK(cudaMemcpyAsync(ctx->boff.p, offsets_host, sizeof(int) * (size_t)(nsys + 1), cudaMemcpyHostToDevice,
                            ctx->stream));
  k_fill_sys<<<nsys, 256, 0, ctx->stream>>>(nsys, P<int>(ctx->boff), P<int>(ctx->bsys));
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  B.S = nsys;
  B.Ntot = N;
  B.off = P<int>(ctx->boff);
  B.sys = P<int>(ctx->bsys);
  B.h_off.assign(offsets_host, offsets_host + nsys + 1);
  return GBI_OK;
}

// ---------------------------------------------------------------------------------
// Tuning of the pair kernel's warps per target
// ---------------------------------------------------------------------------------

// Synthetic timing input: sphere i of system s sits at lattice point i - off[s] of a
// cube of side ceil(cbrt(N_s)) with spacing 3a (so no pair is closer than 3a), and
// every source component is 1e-3.  The pair kernel's work does not depend on values.
__global__ void k_tune_fill(int Ntot, int nsys, const int* __restrict__ off, int* __restrict__ sys_of, double a,
                            float4* __restrict__ hi, float4* __restrict__ lo, double* __restrict__ x, int D) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ntot) return;
  int lo_s = 0, hi_s = nsys - 1;
  while (lo_s < hi_s) {            // last system with off[s] <= i
    const int mid = (lo_s + hi_s + 1) / 2;
    if (off[mid] <= i) lo_s = mid; else hi_s = mid - 1;
  }
  const int s = lo_s;
  sys_of[i] = s;
  const int k = i - off[s], ns = off[s + 1] - off[s];
  int side = 1;
  while (side * side * side < ns) ++side;
  const float sp = float(3.0 * a);
  hi[i] = make_float4(sp * float(k % side), sp * float((k / side) % side), sp * float(k / (side * side)), 0.f);
  lo[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int q = 0; q < D; ++q) x[(size_t)q * Ntot + i] = 1e-3;
}

struct TuneBufs {
  void* p[7] = {};
  ~TuneBufs() {
    for (void* q : p)
      if (q) cudaFree(q);
  }
};

gbi_status tune_impl(gbi_ctx* ctx, int trunc, int nsys, const int* offsets, int reps, int* chosen) {
  const int D = d_of(trunc);
  const int Ntot = offsets[nsys];
  const bool batched = nsys > 1;
  TuneBufs tb;
  const int rf_max = rec_floats(D, true);
  GBI_CHECK(cudaMalloc(&tb.p[0], sizeof(float4) * Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[1], sizeof(float4) * Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[2], sizeof(double) * D * (size_t)Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[3], sizeof(double) * D * (size_t)Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[4], sizeof(float) * rf_max * (size_t)Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[5], sizeof(int) * (size_t)Ntot));
  GBI_CHECK(cudaMalloc(&tb.p[6], sizeof(int) * (size_t)(nsys + 1)));
  float4* hi = static_cast<float4*>(tb.p[0]);
  float4* lo = static_cast<float4*>(tb.p[1]);
  double* x = static_cast<double*>(tb.p[2]);
  double* y = static_cast<double*>(tb.p[3]);
  float* rec = static_cast<float*>(tb.p[4]);
  int* sys_of = static_cast<int*>(tb.p[5]);
  int* sys_off = static_cast<int*>(tb.p[6]);
  GBI_CHECK(cudaMemcpyAsync(sys_off, offsets, sizeof(int) * (nsys + 1), cudaMemcpyHostToDevice, ctx->stream));
  k_tune_fill<<<(Ntot + 255) / 256, 256, 0, ctx->stream>>>(Ntot, nsys, sys_off, sys_of, 1.0, hi, lo, x, D);
  GBI_CHECK(cudaGetLastError());
  ++ctx->launches;
  cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
  struct Pass {
    int rows, cols, precision;
  };
  const Pass passes[4] = {{SET_H, SET_H, 1}, {SET_H, SET_H, 2}, {SET_H, SET_L, 2}, {SET_L, SET_ALL, 2}};
  gbi_status st = GBI_OK;
  for (int k = 0; k < 4 && st == GBI_OK; ++k) {
    const Pass& ps = passes[k];
    PairArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.N = Ntot;
    pa.a = 1.0;
    pa.pos = Positions{hi, lo, nullptr};
    pa.x = x;
    pa.y = y;
    pa.alpha = 1.0;
    for (int i = 0; i < 54; ++i) pa.colscale[i] = 1.0;
    if (batched) {
      pa.sys_of = sys_of;
      pa.sys_off = sys_off;
    }
    const int nc = ncols_of(trunc, ps.cols);
    ColScale cs;
    for (int i = 0; i < 54; ++i) cs.v[i] = 1.0;
    cudaError_t e = launch_records(ps.precision == 2, Ntot, nc, x, nullptr, 0, nullptr, cs, rec, ctx->stream);
    pa.x32 = rec;
    int best = 0;
    float best_ms = 0.f;
    for (int w = 2; w <= max_wpt(trunc, ps.precision) && e == cudaSuccess; w *= 2) {
      pa.wpt = w;
      e = launch_pairs(trunc, ps.rows, ps.cols, ps.precision, pa, ctx->stream);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = launch_pairs(trunc, ps.rows, ps.cols, ps.precision, pa, ctx->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      ctx->launches += 1 + reps;
      if (e == cudaSuccess && (best == 0 || ms < best_ms)) {
        best = w;
        best_ms = ms;
      }
    }
    if (e != cudaSuccess) {
      st = fail(ctx, e, "gbi_tune");
      break;
    }
    ctx->wpt_table[gbi_ctx::wpt_key(trunc, ps.rows, ps.cols, ps.precision, Ntot, batched)] = best;
    if (chosen) chosen[k] = best;
  }
  ctx->pool.push_back(e0);
  ctx->pool.push_back(e1);
  return st;
}


// ---------------------------------------------------------------------------------
// Learned near-field correction: neighbour lists and network driver
// ---------------------------------------------------------------------------------

static_assert(GBI_MLP_NPARAM == mlpk::NPARAM, "flat parameter count");
constexpr int kSmallSystem = 4096;   // one system up to this size: O(N^2) neighbour scan

// Ordered pairs closer than rcut * a within each system, into ctx->nb_* (grouped by
// target, sorted by source).  Reads the pair count back to the host (synchronizes).
gbi_status build_pairs(gbi_ctx* ctx, int N, const double* R, double a, double rcut, int nsys,
                       const int* offsets_host, int& npair) {
  using namespace mlpk;
  const double rc2 = (rcut * a) * (rcut * a);
  const int* sys_of = nullptr;
  const int* sys_off = nullptr;
  Batch B;
  if (nsys > 1) {
    GBI_TRY(make_batch(ctx, nsys, offsets_host, B));
    sys_of = B.sys;
    sys_off = B.off;
  }
  GBI_TRY(ensure(ctx, ctx->nb_cnt, sizeof(int) * (size_t)N));
  GBI_TRY(ensure(ctx, ctx->nb_start, sizeof(int) * (size_t)(N + 1)));
  GBI_TRY(ensure(ctx, ctx->nb_scan, sizeof(int) * scan_scratch_ints(N)));
  GBI_TRY(ensure(ctx, ctx->nb_aux, 64 * 6 * sizeof(double) + 16));
  int* cnt = P<int>(ctx->nb_cnt);
  int* start = P<int>(ctx->nb_start);
  const bool cells = nsys <= 1 && N > kSmallSystem;
  double box[6];
  double side = rcut * a;
  int dims[3] = {1, 1, 1};
  int* overflow = reinterpret_cast<int*>(static_cast<char*>(ctx->nb_aux.p) + 64 * 6 * sizeof(double));
  if (cells) {
    GBI_CHECK(mlpk::bbox(N, R, P<double>(ctx->nb_aux), box, ctx->stream));
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) ext = std::max(ext, box[3 + d] - box[d]);
    side = std::max(side, ext / 96.0);           // at most 97^3 cells
    for (int d = 0; d < 3; ++d) dims[d] = std::max(1, (int)std::ceil((box[3 + d] - box[d]) / side));
    const int nc = dims[0] * dims[1] * dims[2];
    GBI_TRY(ensure(ctx, ctx->cell_of, sizeof(int) * (size_t)N));
    GBI_TRY(ensure(ctx, ctx->cell_cnt, sizeof(int) * (size_t)nc));
    GBI_TRY(ensure(ctx, ctx->cell_start, sizeof(int) * (size_t)nc));
    GBI_TRY(ensure(ctx, ctx->cell_fill, sizeof(int) * (size_t)nc));
    GBI_TRY(ensure(ctx, ctx->cell_items, sizeof(int) * (size_t)N));
    if (ensure(ctx, ctx->nb_scan, sizeof(int) * std::max(scan_scratch_ints(N), scan_scratch_ints(nc))) != GBI_OK)
      return GBI_ERR_NOMEM;
    GBI_CHECK(cells_build(N, R, box, side, dims, P<int>(ctx->cell_of), P<int>(ctx->cell_cnt),
                          P<int>(ctx->cell_start), P<int>(ctx->cell_fill), P<int>(ctx->cell_items),
                          P<int>(ctx->nb_scan), ctx->stream));
    GBI_CHECK(cudaMemsetAsync(overflow, 0, sizeof(int), ctx->stream));
    GBI_CHECK(nb_cells(N, R, box, side, dims, P<int>(ctx->cell_of), P<int>(ctx->cell_start), P<int>(ctx->cell_cnt),
                       P<int>(ctx->cell_items), rc2, nullptr, cnt, nullptr, nullptr, overflow, ctx->stream));
    ctx->launches += 6;
  } else {
    GBI_CHECK(nb_count_sys(N, R, sys_of, sys_off, rc2, cnt, ctx->stream));
    ++ctx->launches;
  }
  GBI_CHECK(exclusive_scan(cnt, start, N, P<int>(ctx->nb_scan), ctx->stream));
  ctx->launches += 3;
  const int chunks = (N + 1023) / 1024;
  int total = 0, ovf = 0;
  GBI_CHECK(cudaMemcpyAsync(&total, P<int>(ctx->nb_scan) + chunks, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  if (cells) GBI_CHECK(cudaMemcpyAsync(&ovf, overflow, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GBI_CHECK(cudaMemcpyAsync(start + N, P<int>(ctx->nb_scan) + chunks, sizeof(int), cudaMemcpyDeviceToDevice,
                            ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  if (ovf) {
    ctx->err = "more than 64 neighbours within the cut-off for some sphere (overlapping input?)";
    return GBI_ERR_ARG;
  }
  GBI_TRY(ensure(ctx, ctx->nb_tg, sizeof(int) * (size_t)std::max(total, 1)));
  GBI_TRY(ensure(ctx, ctx->nb_sr, sizeof(int) * (size_t)std::max(total, 1)));
  if (cells)
    GBI_CHECK(nb_cells(N, R, box, side, dims, P<int>(ctx->cell_of), P<int>(ctx->cell_start), P<int>(ctx->cell_cnt),
                       P<int>(ctx->cell_items), rc2, start, nullptr, P<int>(ctx->nb_tg), P<int>(ctx->nb_sr), overflow,
                       ctx->stream));
  else
    GBI_CHECK(nb_fill_sys(N, R, sys_of, sys_off, rc2, start, P<int>(ctx->nb_tg), P<int>(ctx->nb_sr), ctx->stream));
  ++ctx->launches;
  ctx->nb_pairs = total;
  ctx->nb_N = N;
  npair = total;
  return GBI_OK;
}

gbi_status mlp_require(gbi_ctx* ctx) {
  if (!ctx->mlp_ready) {
    ctx->err = "no network loaded (gbi_mlp_set)";
    return GBI_ERR_ARG;
  }
  return GBI_OK;
}

// pairs (rcut 4a) and their features for N spheres; returns the pair count
gbi_status mlp_prepare(gbi_ctx* ctx, int N, const double* R, const double* p, double a, int nsys,
                       const int* offsets_host, int& npair) {
  GBI_TRY(build_pairs(ctx, N, R, a, 4.0, nsys, offsets_host, npair));
  const size_t n = (size_t)std::max(npair, 1);
  GBI_TRY(ensure(ctx, ctx->mf_F, sizeof(float) * mlpk::NIN * n));
  GBI_TRY(ensure(ctx, ctx->mf_FR, sizeof(float) * 9 * n));
  GBI_TRY(ensure(ctx, ctx->mf_lab, sizeof(float) * 6 * n));
  GBI_CHECK(mlpk::features(npair, R, p, P<int>(ctx->nb_tg), P<int>(ctx->nb_sr), a, P<float>(ctx->mf_F),
                           P<float>(ctx->mf_FR), ctx->stream));
  ++ctx->launches;
  return GBI_OK;
}

int sm_count(gbi_ctx* ctx) {
  if (ctx->num_sms == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || v <= 0) v = 152;
    ctx->num_sms = v;
  }
  return ctx->num_sms;
}

// Network inference with the selected engine.  The tcgen05 kernel reports a wait that
// gave up through a device flag that gbi_mlp_status reads back.
gbi_status mlp_infer(gbi_ctx* ctx, int np_, const float* F, const float* FR, float* out) {
  if (ctx->mlp_engine == 1) {
    GBI_CHECK(mlpk::infer_tc(np_, F, FR, ctx->mlp_pk_tc.p, out, P<int>(ctx->mlp_err), sm_count(ctx), ctx->stream));
    ++ctx->launches;
    return GBI_OK;
  }
  GBI_CHECK(mlpk::infer(np_, F, FR, ctx->mlp_pk.p, out, sm_count(ctx), ctx->stream));
  ++ctx->launches;
  return GBI_OK;
}

}  // namespace

// =================================================================================
// C ABI
// =================================================================================

extern "C" {

gbi_status gbi_create(gbi_ctx** out, int device) {
  if (!out) return GBI_ERR_ARG;
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return GBI_ERR_CUDA;
  gbi_ctx* c = new gbi_ctx();
  c->device = device;
  e = cudaMallocHost(&c->hbuf, sizeof(double) * (2 * kMaxRestart + 16));
  if (e != cudaSuccess) {
    delete c;
    return GBI_ERR_NOMEM;
  }
  *out = c;
  return GBI_OK;
}

gbi_status gbi_destroy(gbi_ctx* ctx) {
  if (!ctx) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  Buf* bufs[] = {&ctx->pos_hi, &ctx->pos_lo, &ctx->pos64, &ctx->xF, &ctx->xVH, &ctx->b, &ctx->xQ, &ctx->r,
                 &ctx->delta, &ctx->krylov, &ctx->w, &ctx->partial, &ctx->dots, &ctx->xVL, &ctx->minr2,
                 &ctx->colbuf, &ctx->x32, &ctx->trapbuf, &ctx->gstate, &ctx->boff, &ctx->bsys, &ctx->tFe, &ctx->tTe, &ctx->tVa, &ctx->tOa, &ctx->tVH, &ctx->tV, &ctx->tOm,
                 &ctx->tQH, &ctx->hR, &ctx->hVa, &ctx->hOa, &ctx->hVH, &ctx->hFe, &ctx->hTe, &ctx->hV,
                 &ctx->hOm, &ctx->hQH, &ctx->mlp_th, &ctx->mlp_m, &ctx->mlp_v, &ctx->mlp_thq, &ctx->mlp_pk,
                 &ctx->mlp_grad, &ctx->mlp_pk_tc, &ctx->mlp_err, &ctx->nb_cnt, &ctx->nb_start, &ctx->nb_tg, &ctx->nb_sr, &ctx->nb_scan,
                 &ctx->cell_of, &ctx->cell_cnt, &ctx->cell_start, &ctx->cell_fill, &ctx->cell_items, &ctx->nb_aux,
                 &ctx->mf_F, &ctx->mf_FR, &ctx->mf_lab, &ctx->mf_dO, &ctx->mf_part, &ctx->mf_loss};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (ctx->hbuf) cudaFreeHost(ctx->hbuf);
  drain_profile(ctx);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  if (ctx->chunk_exec) cudaGraphExecDestroy(ctx->chunk_exec);
  delete ctx;
  return GBI_OK;
}

gbi_status gbi_set_stream(gbi_ctx* ctx, void* stream) {
  if (!ctx) return GBI_ERR_ARG;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  return GBI_OK;
}

gbi_status gbi_synchronize(gbi_ctx* ctx) {
  if (!ctx) return GBI_ERR_ARG;
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  return GBI_OK;
}

const char* gbi_status_string(int status) {
  switch (status) {
    case GBI_OK: return "ok";
    case GBI_ERR_ARG: return "invalid argument";
    case GBI_ERR_OVERLAP: return "spheres overlap (closer than min_sep * a)";
    case GBI_ERR_NOT_CONVERGED: return "iteration cap reached before the tolerance";
    case GBI_ERR_TIMEOUT: return "bounded device wait gave up";
    case GBI_ERR_CUDA: return "CUDA runtime error";
    case GBI_ERR_NOMEM: return "workspace allocation failed";
    default: return "unknown status";
  }
}

const char* gbi_last_error(gbi_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

int gbi_h(int trunc) { return d_of(trunc) < 0 ? -1 : d_of(trunc) - 6; }
int gbi_d(int trunc) { return d_of(trunc); }

gbi_status gbi_component_scales(int trunc, double* out_host) {
  if (d_of(trunc) < 0 || !out_host) return GBI_ERR_ARG;
  std::memcpy(out_host, scale_tab(trunc), sizeof(double) * d_of(trunc));
  return GBI_OK;
}

gbi_status gbi_self_scalars(int trunc, double* out_host) {
  if (d_of(trunc) < 0 || !out_host) return GBI_ERR_ARG;
  std::memcpy(out_host, self_tab(trunc), sizeof(double) * d_of(trunc));
  return GBI_OK;
}

gbi_status gbi_apply(gbi_ctx* ctx, int N, int trunc, double a, int rows, int cols, int precision,
                     const double* R, const double* x, double* y, double alpha, double beta, int add_self) {
  if (!ctx || N < 0 || d_of(trunc) < 0 || !(a > 0) || precision < 0 || precision > 2) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !x || !y) return GBI_ERR_ARG;
  const bool supported = (rows == SET_H && cols == SET_L) || (rows == SET_H && cols == SET_H) ||
                         (rows == SET_L && cols == SET_ALL) || (rows == SET_ALL && cols == SET_ALL);
  if (!supported) return GBI_ERR_ARG;
  if (precision == 2 && rows == SET_ALL && cols == SET_ALL) return GBI_ERR_ARG;
  if (add_self && rows != cols && !(rows == SET_L && cols == SET_ALL)) return GBI_ERR_ARG;
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, trunc, a, 1.0, R));
  PairArgs p = pair_args(s, x, y, alpha, beta, add_self, s.ones, 0);
  GBI_CHECK(run_pairs(ctx, trunc, rows, cols, precision, p));
  return GBI_OK;
}

gbi_status gbi_solve(gbi_ctx* ctx, const gbi_params* prm, int N, const double* R, const double* Va,
                     const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                     double* Omega, double* QH, int warm_start, gbi_info* info) {
  if (!ctx || !valid_params(prm) || N < 0) return GBI_ERR_ARG;
  gbi_info local{};
  gbi_info* inf = info ? info : &local;
  *inf = gbi_info{};
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega || (warm_start && !QH)) return GBI_ERR_ARG;
  Batch B;
  GBI_TRY(single_batch(ctx, N, B));
  return solve_core(ctx, prm, B, R, Va, Oa, VH, Fe, Te, V, Omega, QH, warm_start, inf);
}

gbi_status gbi_batch_solve(gbi_ctx* ctx, const gbi_params* prm, int nsys, const int* offsets_host, const double* R,
                           const double* Va, const double* Oa, const double* VH, const double* Fe, const double* Te,
                           double* V, double* Omega, double* QH, int warm_start, gbi_info* info) {
  if (!ctx || !valid_params(prm) || nsys < 0 || (nsys > 0 && !offsets_host)) return GBI_ERR_ARG;
  gbi_info local{};
  gbi_info* inf = info ? info : &local;
  *inf = gbi_info{};
  if (nsys == 0) return GBI_OK;
  if (!valid_offsets(nsys, offsets_host)) return GBI_ERR_ARG;
  const int N = offsets_host[nsys];
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega || (warm_start && !QH)) return GBI_ERR_ARG;
  Batch B;
  GBI_TRY(make_batch(ctx, nsys, offsets_host, B));
  return solve_core(ctx, prm, B, R, Va, Oa, VH, Fe, Te, V, Omega, QH, warm_start, inf);
}

gbi_status gbi_batch_superpose(gbi_ctx* ctx, const gbi_params* prm, int nsys, const int* offsets_host,
                               const double* R, const double* Va, const double* Oa, const double* VH,
                               const double* Fe, const double* Te, double* V, double* Omega) {
  if (!ctx || !valid_params(prm) || nsys < 0 || (nsys > 0 && !offsets_host)) return GBI_ERR_ARG;
  if (nsys == 0) return GBI_OK;
  if (!valid_offsets(nsys, offsets_host)) return GBI_ERR_ARG;
  const int N = offsets_host[nsys];
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega) return GBI_ERR_ARG;
  Batch B;
  GBI_TRY(make_batch(ctx, nsys, offsets_host, B));
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, prm->trunc, prm->a, prm->eta, R));
  const int D = s.D, h = s.h;
  const size_t nh = (size_t)N * h;
  GBI_TRY(ensure(ctx, ctx->xQ, sizeof(double) * (size_t)N * D));
  GBI_TRY(ensure(ctx, ctx->xVL, sizeof(double) * 6 * N));
  double* xF = P<double>(ctx->xQ);
  double* xQH = P<double>(ctx->xQ) + (size_t)6 * N;
  Scales oneb;   // one-body Q^H = -8 pi eta a V^H / g, in internal coordinates
  for (int i = 0; i < 54; ++i) oneb.v[i] = (i < h) ? s.scale.v[6 + i] * s.a / s.selfg.v[6 + i] : 1.0;
  k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], Fe, Te, xF);
  ++ctx->launches;
  k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, oneb, -8.0 * kPi * s.eta, xQH);
  ++ctx->launches;
  PairArgs p = pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1, s.ones,
                         0);
  p.sys_of = B.sys;
  p.sys_off = B.off;
  GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, prm->precision == 3 ? 1 : prm->precision, p));
  k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], P<double>(ctx->xVL), Va, Oa, V,
                                                      Omega);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_superpose(gbi_ctx* ctx, const gbi_params* prm, int N, const double* R, const double* Va,
                         const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                         double* Omega) {
  if (!ctx || !valid_params(prm) || N < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega) return GBI_ERR_ARG;
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, prm->trunc, prm->a, prm->eta, R));
  if (prm->trunc == 2) {
    TrapArgs t;
    t.N = N;
    t.a = prm->a;
    t.eta = prm->eta;
    t.pos = s.pos;
    t.Fe = Fe;
    t.Te = Te;
    t.VH = VH;
    t.Va = Va;
    t.Oa = Oa;
    t.V = V;
    t.Om = Omega;
    GBI_CHECK(run_trap(ctx, t, prm->precision == 3 ? 1 : prm->precision));
    return GBI_OK;
  }
  const int D = s.D, h = s.h;
  const size_t nh = (size_t)N * h;
  GBI_TRY(ensure(ctx, ctx->xQ, sizeof(double) * (size_t)N * D));
  GBI_TRY(ensure(ctx, ctx->xVL, sizeof(double) * 6 * N));
  double* xF = P<double>(ctx->xQ);
  double* xQH = P<double>(ctx->xQ) + (size_t)6 * N;
  Scales oneb;   // one-body Q^H = -8 pi eta a V^H / g, in internal coordinates
  for (int i = 0; i < 54; ++i) oneb.v[i] = (i < h) ? s.scale.v[6 + i] * s.a / s.selfg.v[6 + i] : 1.0;
  k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], Fe, Te, xF);
  ++ctx->launches;
  k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, oneb, -8.0 * kPi * s.eta, xQH);
  ++ctx->launches;
  PairArgs p = pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1, s.ones,
                         0);
  GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, prm->precision == 3 ? 1 : prm->precision, p));
  k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], P<double>(ctx->xVL), Va, Oa, V,
                                                      Omega);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_trap_step(gbi_ctx* ctx, const gbi_params* prm, int N, double dt, double k_trap, double vs,
                         double s0, double d0, int superposition, int nsteps, double* R, double* p,
                         gbi_info* info) {
  if (!ctx || !valid_params(prm) || N < 0 || nsteps < 0) return GBI_ERR_ARG;
  gbi_info total{};
  if (N == 0 || nsteps == 0) {
    if (info) *info = total;
    return GBI_OK;
  }
  if (!R || !p) return GBI_ERR_ARG;
  const int h = gbi_h(prm->trunc);
  GBI_TRY(ensure(ctx, ctx->tFe, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tTe, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tVa, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tOa, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tVH, sizeof(double) * (size_t)h * N));
  GBI_TRY(ensure(ctx, ctx->tV, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tOm, sizeof(double) * 3 * N));
  GBI_TRY(ensure(ctx, ctx->tQH, sizeof(double) * (size_t)h * N));
  gbi_status st = GBI_OK;
  for (int step = 0; step < nsteps; ++step) {
    k_trap_inputs<<<grid1(N), 256, 0, ctx->stream>>>(N, k_trap, vs, s0, d0, h, R, p, P<double>(ctx->tFe),
                                                     P<double>(ctx->tTe), P<double>(ctx->tVa), P<double>(ctx->tOa),
                                                     P<double>(ctx->tVH));
    ++ctx->launches;
    GBI_CHECK(cudaGetLastError());
    if (superposition) {
      GBI_TRY(gbi_superpose(ctx, prm, N, R, P<double>(ctx->tVa), P<double>(ctx->tOa), P<double>(ctx->tVH),
                            P<double>(ctx->tFe), P<double>(ctx->tTe), P<double>(ctx->tV), P<double>(ctx->tOm)));
      total.pair_interactions += (long long)N * (N - 1);
      (prm->precision == 1 || prm->precision == 3 ? total.matvecs_f32 : total.matvecs_f64) += 1;
    } else {
      gbi_info one{};
      // FP64 solves warm-start from the previous step's traction coefficients (also across
      // calls with the same N and truncation on this context).  Mixed-precision solves start
      // from zero: a warm start costs one more high-precision residual pass, and the FP32
      // inner solves cannot reach the target from it in fewer sweeps.
      const bool warm = prm->precision == 0 && (step > 0 || (ctx->tqh_N == N && ctx->tqh_trunc == prm->trunc));
      ctx->tqh_N = -1;
      st = gbi_solve(ctx, prm, N, R, P<double>(ctx->tVa), P<double>(ctx->tOa), P<double>(ctx->tVH),
                     P<double>(ctx->tFe), P<double>(ctx->tTe), P<double>(ctx->tV), P<double>(ctx->tOm),
                     P<double>(ctx->tQH), warm ? 1 : 0, &one);
      if (st == GBI_OK) {
        ctx->tqh_N = N;
        ctx->tqh_trunc = prm->trunc;
      }
      total.iters += one.iters;
      total.refinements += one.refinements;
      total.matvecs_f32 += one.matvecs_f32;
      total.matvecs_f64 += one.matvecs_f64;
      total.pair_interactions += one.pair_interactions;
      total.rel_residual = std::max(total.rel_residual, one.rel_residual);
      total.min_separation = step == 0 ? one.min_separation : std::min(total.min_separation, one.min_separation);
      if (st != GBI_OK) break;
    }
    k_euler<<<grid1(N), 256, 0, ctx->stream>>>(N, dt, P<double>(ctx->tV), P<double>(ctx->tOm), R, p);
    ++ctx->launches;
    GBI_CHECK(cudaGetLastError());
  }
  if (info) *info = total;
  return st;
}

gbi_status gbi_trap_inputs(gbi_ctx* ctx, int N, int trunc, double k_trap, double vs, double s0, double d0,
                           const double* R, const double* p, double* Fe, double* Te, double* Va, double* Oa,
                           double* VH) {
  if (!ctx || N < 0 || d_of(trunc) < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !p || !Fe || !Te || !Va || !Oa || !VH) return GBI_ERR_ARG;
  k_trap_inputs<<<grid1(N), 256, 0, ctx->stream>>>(N, k_trap, vs, s0, d0, gbi_h(trunc), R, p, Fe, Te, Va, Oa, VH);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_tune(gbi_ctx* ctx, int trunc, int nsys, const int* offsets, int reps, int* chosen) {
  if (!ctx || d_of(trunc) < 0 || nsys < 1 || !offsets || reps < 0) return GBI_ERR_ARG;
  if (offsets[0] != 0) return GBI_ERR_ARG;
  for (int s = 0; s < nsys; ++s)
    if (offsets[s + 1] <= offsets[s]) return GBI_ERR_ARG;
  if (reps == 0) reps = 5;
  return tune_impl(ctx, trunc, nsys, offsets, reps, chosen);
}

gbi_status gbi_set_wpt(gbi_ctx* ctx, int wpt) {
  if (!ctx || !(wpt == 0 || wpt == 2 || wpt == 4 || wpt == 8 || wpt == 16)) return GBI_ERR_ARG;
  ctx->force_wpt = wpt;
  return GBI_OK;
}

int gbi_pass_wpt(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, int N, int batched) {
  if (!ctx || d_of(trunc) < 0 || rows < 0 || rows > 2 || cols < 0 || cols > 2 || N < 1) return -1;
  if (precision == 0) return 0;
  if (precision != 1 && precision != 2) return -1;
  const int req = ctx->force_wpt > 0 ? ctx->force_wpt : ctx->tuned_wpt(trunc, rows, cols, precision, N, batched != 0);
  return stream_wpt(trunc, precision, N, req);
}

gbi_status gbi_pairs(gbi_ctx* ctx, int N, const double* R, double a, double rcut, int nsys, const int* offsets_host,
                     int* npairs) {
  if (!ctx || N < 0 || !(a > 0) || !(rcut > 0) || nsys < 0 || (nsys > 1 && !offsets_host)) return GBI_ERR_ARG;
  if (nsys > 1 && (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N)) return GBI_ERR_ARG;
  if (N == 0) {
    ctx->nb_pairs = 0;
    if (npairs) *npairs = 0;
    return GBI_OK;
  }
  if (!R) return GBI_ERR_ARG;
  int np_ = 0;
  GBI_TRY(build_pairs(ctx, N, R, a, rcut, nsys, offsets_host, np_));
  if (npairs) *npairs = np_;
  return GBI_OK;
}

gbi_status gbi_pairs_get(gbi_ctx* ctx, int* tg, int* sr) {
  if (!ctx) return GBI_ERR_ARG;
  if (ctx->nb_pairs == 0) return GBI_OK;
  if (!tg || !sr) return GBI_ERR_ARG;
  GBI_CHECK(cudaMemcpyAsync(tg, ctx->nb_tg.p, sizeof(int) * (size_t)ctx->nb_pairs, cudaMemcpyDeviceToDevice,
                            ctx->stream));
  GBI_CHECK(cudaMemcpyAsync(sr, ctx->nb_sr.p, sizeof(int) * (size_t)ctx->nb_pairs, cudaMemcpyDeviceToDevice,
                            ctx->stream));
  return GBI_OK;
}

gbi_status gbi_mlp_set(gbi_ctx* ctx, const float* theta_host, double sigma) {
  if (!ctx || !theta_host || !(sigma > 0)) return GBI_ERR_ARG;
  const size_t nb = sizeof(float) * mlpk::NPARAM;
  GBI_TRY(ensure(ctx, ctx->mlp_th, nb));
  GBI_TRY(ensure(ctx, ctx->mlp_m, nb));
  GBI_TRY(ensure(ctx, ctx->mlp_v, nb));
  GBI_TRY(ensure(ctx, ctx->mlp_thq, nb));
  GBI_TRY(ensure(ctx, ctx->mlp_grad, nb));
  GBI_TRY(ensure(ctx, ctx->mlp_pk, mlpk::packed_bytes()));
  GBI_TRY(ensure(ctx, ctx->mlp_pk_tc, mlpk::packed_tc_bytes()));
  GBI_TRY(ensure(ctx, ctx->mlp_err, sizeof(int)));
  GBI_CHECK(cudaMemsetAsync(ctx->mlp_err.p, 0, sizeof(int), ctx->stream));
  GBI_CHECK(cudaMemcpyAsync(ctx->mlp_th.p, theta_host, nb, cudaMemcpyHostToDevice, ctx->stream));
  GBI_CHECK(cudaMemsetAsync(ctx->mlp_m.p, 0, nb, ctx->stream));
  GBI_CHECK(cudaMemsetAsync(ctx->mlp_v.p, 0, nb, ctx->stream));
  GBI_CHECK(mlpk::pack_weights(P<float>(ctx->mlp_th), P<float>(ctx->mlp_thq), ctx->mlp_pk.p, ctx->stream));
  GBI_CHECK(mlpk::pack_weights_tc(P<float>(ctx->mlp_th), ctx->mlp_pk_tc.p, ctx->stream));
  ctx->launches += 2;
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));   // theta_host may be reused by the caller
  ctx->mlp_sigma = sigma;
  ctx->mlp_step = 0;
  ctx->mlp_ready = true;
  return GBI_OK;
}

gbi_status gbi_mlp_get(gbi_ctx* ctx, float* theta_host, double* sigma) {
  if (!ctx || !theta_host) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  GBI_CHECK(cudaMemcpyAsync(theta_host, ctx->mlp_th.p, sizeof(float) * mlpk::NPARAM, cudaMemcpyDeviceToHost,
                            ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  if (sigma) *sigma = ctx->mlp_sigma;
  return GBI_OK;
}

gbi_status gbi_mlp_features(gbi_ctx* ctx, int P, const double* R, const double* p, const int* tg, const int* sr,
                            double a, float* F, float* FR) {
  if (!ctx || P < 0 || !(a > 0)) return GBI_ERR_ARG;
  if (P == 0) return GBI_OK;
  if (!R || !p || !tg || !sr || !F || !FR) return GBI_ERR_ARG;
  GBI_CHECK(mlpk::features(P, R, p, tg, sr, a, F, FR, ctx->stream));
  ++ctx->launches;
  return GBI_OK;
}

gbi_status gbi_mlp_forward(gbi_ctx* ctx, int P, const float* F, const float* FR, float* out) {
  if (!ctx || P < 0) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  if (P == 0) return GBI_OK;
  if (!F || !out) return GBI_ERR_ARG;
  return mlp_infer(ctx, P, F, FR, out);
}

gbi_status gbi_mlp_status(gbi_ctx* ctx) {
  if (!ctx) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  int e = 0;
  GBI_CHECK(cudaMemcpyAsync(&e, ctx->mlp_err.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  if (e) {
    GBI_CHECK(cudaMemsetAsync(ctx->mlp_err.p, 0, sizeof(int), ctx->stream));
    ctx->err = "tensor-core inference: an MMA completion wait gave up";
    return GBI_ERR_TIMEOUT;
  }
  return GBI_OK;
}

gbi_status gbi_mlp_set_engine(gbi_ctx* ctx, int engine) {
  if (!ctx || engine < 0 || engine > 1) return GBI_ERR_ARG;
  ctx->mlp_engine = engine;
  return GBI_OK;
}

gbi_status gbi_mlp_correct(gbi_ctx* ctx, int N, const double* R, const double* p, double a, double s0, int nsys,
                           const int* offsets_host, double* V, double* Omega, int* npairs) {
  if (!ctx || N < 0 || !(a > 0) || nsys < 0 || (nsys > 1 && !offsets_host)) return GBI_ERR_ARG;
  if (nsys > 1 && (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N)) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  if (npairs) *npairs = 0;
  if (N == 0) return GBI_OK;
  if (!R || !p || !V || !Omega) return GBI_ERR_ARG;
  int np_ = 0;
  GBI_TRY(mlp_prepare(ctx, N, R, p, a, nsys, offsets_host, np_));
  GBI_TRY(mlp_infer(ctx, np_, P<float>(ctx->mf_F), P<float>(ctx->mf_FR), P<float>(ctx->mf_lab)));
  GBI_CHECK(mlpk::sphere_sums(N, P<int>(ctx->nb_start), P<float>(ctx->mf_lab), s0 / ctx->mlp_sigma, V, Omega,
                              ctx->stream));
  ctx->launches += 1;
  if (npairs) *npairs = np_;
  return GBI_OK;
}

gbi_status gbi_mlp_loss_grad(gbi_ctx* ctx, int N, const double* R, const double* p, double a, int nsys,
                             const int* offsets_host, const double* labels, double* loss, float* grad) {
  if (!ctx || N <= 0 || !(a > 0) || nsys < 0 || (nsys > 1 && !offsets_host)) return GBI_ERR_ARG;
  if (nsys > 1 && (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N)) return GBI_ERR_ARG;
  if (!R || !p || !labels || !loss || !grad) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  int np_ = 0;
  GBI_TRY(mlp_prepare(ctx, N, R, p, a, nsys, offsets_host, np_));
  const size_t n = (size_t)std::max(np_, 1);
  GBI_TRY(ensure(ctx, ctx->mf_dO, sizeof(float) * 6 * n));
  GBI_TRY(ensure(ctx, ctx->mf_part, sizeof(float) * std::max<size_t>(mlpk::train_part_floats(np_), 1)));
  const int nlb = (N + 127) / 128;
  GBI_TRY(ensure(ctx, ctx->mf_loss, sizeof(double) * (size_t)(nlb + 1)));
  GBI_CHECK(mlpk::train_batch(P<float>(ctx->mlp_thq), P<float>(ctx->mf_F), P<float>(ctx->mf_FR),
                              P<int>(ctx->nb_start), labels, 0, np_, 0, N, N, P<float>(ctx->mf_lab),
                              P<float>(ctx->mf_dO), P<float>(ctx->mf_part), P<double>(ctx->mf_loss), grad,
                              ctx->stream));
  GBI_CHECK(mlpk::sum_into(P<double>(ctx->mf_loss), nlb, P<double>(ctx->mf_loss) + nlb, ctx->stream));
  ctx->launches += 5;
  GBI_CHECK(cudaMemcpyAsync(loss, P<double>(ctx->mf_loss) + nlb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  return GBI_OK;
}

gbi_status gbi_mlp_adam(gbi_ctx* ctx, const float* grad, double lr) {
  if (!ctx || !grad || !(lr >= 0)) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  ++ctx->mlp_step;
  GBI_CHECK(mlpk::adam(P<float>(ctx->mlp_th), P<float>(ctx->mlp_m), P<float>(ctx->mlp_v), grad, ctx->mlp_step, lr,
                       P<float>(ctx->mlp_thq), ctx->mlp_pk.p, ctx->mlp_pk_tc.p, ctx->stream));
  ctx->launches += 3;
  return GBI_OK;
}

gbi_status gbi_mlp_labels(gbi_ctx* ctx, int N, double s0, const double* Vx, const double* Ox, const double* Vs,
                          const double* Os, double* sigma, double* labels) {
  if (!ctx || N <= 0 || !(s0 != 0) || !Vx || !Ox || !Vs || !Os || !sigma || !labels) return GBI_ERR_ARG;
  if (!(*sigma > 0)) {
    // sigma = the power of two nearest to 1 / rms of (exact - superposition) / s0
    const int nb = (N + 255) / 256;
    GBI_TRY(ensure(ctx, ctx->mf_loss, sizeof(double) * (size_t)(nb + 1)));
    GBI_CHECK(mlpk::labels(N, s0, 1.0, Vx, Ox, Vs, Os, nullptr, P<double>(ctx->mf_loss), ctx->stream));
    GBI_CHECK(mlpk::sum_into(P<double>(ctx->mf_loss), nb, P<double>(ctx->mf_loss) + nb, ctx->stream));
    ctx->launches += 2;
    double sq = 0.0;
    GBI_CHECK(cudaMemcpyAsync(&sq, P<double>(ctx->mf_loss) + nb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    const double rms = std::sqrt(sq / (6.0 * N));
    if (!(rms > 0)) return GBI_ERR_ARG;
    *sigma = std::ldexp(1.0, (int)std::lround(-std::log2(rms)));
  }
  GBI_CHECK(mlpk::labels(N, s0, *sigma, Vx, Ox, Vs, Os, labels, nullptr, ctx->stream));
  ++ctx->launches;
  return GBI_OK;
}

gbi_status gbi_mlp_train(gbi_ctx* ctx, int N, const double* R, const double* p, double a, int nsys,
                         const int* offsets_host, const double* labels, int epochs, int batch_systems, double lr0,
                         double lr1, double* loss_hist) {
  if (!ctx || N <= 0 || !(a > 0) || nsys < 1 || !offsets_host || epochs < 0 || batch_systems < 1 || !(lr0 > 0) ||
      !(lr1 > 0))
    return GBI_ERR_ARG;
  if (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N) return GBI_ERR_ARG;
  if (!R || !p || !labels) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  int np_ = 0;
  GBI_TRY(mlp_prepare(ctx, N, R, p, a, nsys, offsets_host, np_));
  std::vector<int> hstart(N + 1);
  GBI_CHECK(cudaMemcpyAsync(hstart.data(), ctx->nb_start.p, sizeof(int) * (size_t)(N + 1), cudaMemcpyDeviceToHost,
                            ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  const int nbatch = (nsys + batch_systems - 1) / batch_systems;
  int max_pairs = 1, max_spheres = 1;
  for (int b = 0; b < nbatch; ++b) {
    const int s0 = b * batch_systems, s1 = std::min(nsys, s0 + batch_systems);
    max_pairs = std::max(max_pairs, hstart[offsets_host[s1]] - hstart[offsets_host[s0]]);
    max_spheres = std::max(max_spheres, offsets_host[s1] - offsets_host[s0]);
  }
  const size_t n = (size_t)std::max(np_, 1);
  GBI_TRY(ensure(ctx, ctx->mf_dO, sizeof(float) * 6 * n));
  GBI_TRY(ensure(ctx, ctx->mf_part, sizeof(float) * mlpk::train_part_floats(max_pairs)));
  const int nlb = (max_spheres + 127) / 128;
  GBI_TRY(ensure(ctx, ctx->mf_loss, sizeof(double) * (size_t)(nlb + nbatch)));
  double* lpart = P<double>(ctx->mf_loss);
  double* lstep = lpart + nlb;
  const long long total_steps = (long long)epochs * nbatch;
  long long step = 0;
  std::vector<double> hl(nbatch);
  for (int e = 0; e < epochs; ++e) {
    for (int b = 0; b < nbatch; ++b, ++step) {
      const int s0 = b * batch_systems, s1 = std::min(nsys, s0 + batch_systems);
      const int n0 = offsets_host[s0], n1 = offsets_host[s1];
      GBI_CHECK(mlpk::train_batch(P<float>(ctx->mlp_thq), P<float>(ctx->mf_F), P<float>(ctx->mf_FR),
                                  P<int>(ctx->nb_start), labels, hstart[n0], hstart[n1], n0, n1, n1 - n0,
                                  P<float>(ctx->mf_lab), P<float>(ctx->mf_dO), P<float>(ctx->mf_part), lpart,
                                  P<float>(ctx->mlp_grad), ctx->stream));
      GBI_CHECK(mlpk::sum_into(lpart, (n1 - n0 + 127) / 128, lstep + b, ctx->stream));
      // learning rate: geometric from lr0 to lr1 over all steps
      const double frac = total_steps > 1 ? double(step) / double(total_steps - 1) : 0.0;
      const double lr = lr0 * std::pow(lr1 / lr0, frac);
      ++ctx->mlp_step;
      GBI_CHECK(mlpk::adam(P<float>(ctx->mlp_th), P<float>(ctx->mlp_m), P<float>(ctx->mlp_v),
                           P<float>(ctx->mlp_grad), ctx->mlp_step, lr, P<float>(ctx->mlp_thq), ctx->mlp_pk.p,
                           ctx->mlp_pk_tc.p, ctx->stream));
      ctx->launches += 8;
    }
    GBI_CHECK(cudaMemcpyAsync(hl.data(), lstep, sizeof(double) * nbatch, cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    if (loss_hist) {
      double acc = 0.0;
      for (double v : hl) acc += v;
      loss_hist[e] = acc / nbatch;
    }
  }
  return GBI_OK;
}

gbi_status gbi_set_profiling(gbi_ctx* ctx, int on) {
  if (!ctx) return GBI_ERR_ARG;
  drain_profile(ctx);
  ctx->prof = on != 0;
  for (int i = 0; i < 30; ++i) {
    ctx->stat_dead[i] = 0;
    ctx->stat_ms[i] = 0.0;
    ctx->stat_flops[i] = 0.0;
    ctx->stat_n[i] = 0;
  }
  return GBI_OK;
}

gbi_status gbi_kernel_stats(gbi_ctx* ctx, int kernel_class, double* total_ms, long long* launches,
                            double* flops) {
  if (!ctx || kernel_class < 0 || kernel_class >= 30) return GBI_ERR_ARG;
  drain_profile(ctx);
  if (total_ms) *total_ms = ctx->stat_ms[kernel_class];
  const long long live = ctx->stat_n[kernel_class] - (ctx->prof ? ctx->stat_dead[kernel_class] : 0);
  const double per = ctx->stat_n[kernel_class] > 0 ? ctx->stat_flops[kernel_class] / ctx->stat_n[kernel_class] : 0.0;
  if (launches) *launches = live;
  if (flops) *flops = per * double(live);
  return GBI_OK;
}

long long gbi_kernel_launches(gbi_ctx* ctx) { return ctx ? ctx->launches : -1; }

gbi_status gbi_solve_host(gbi_ctx* ctx, const gbi_params* prm, int N, const double* R, const double* Va,
                          const double* Oa, const double* VH, const double* Fe, const double* Te, double* V,
                          double* Omega, double* QH, int warm_start, gbi_info* info) {
  if (!ctx || !valid_params(prm) || N < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega || (warm_start && !QH)) return GBI_ERR_ARG;
  const int h = gbi_h(prm->trunc);
  const size_t v3 = sizeof(double) * 3 * N, vh = sizeof(double) * (size_t)h * N;
  GBI_TRY(ensure(ctx, ctx->hR, v3));
  GBI_TRY(ensure(ctx, ctx->hVa, v3));
  GBI_TRY(ensure(ctx, ctx->hOa, v3));
  GBI_TRY(ensure(ctx, ctx->hVH, vh));
  GBI_TRY(ensure(ctx, ctx->hFe, v3));
  GBI_TRY(ensure(ctx, ctx->hTe, v3));
  GBI_TRY(ensure(ctx, ctx->hV, v3));
  GBI_TRY(ensure(ctx, ctx->hOm, v3));
  GBI_TRY(ensure(ctx, ctx->hQH, vh));
  cudaStream_t st = ctx->stream;
  GBI_CHECK(cudaMemcpyAsync(ctx->hR.p, R, v3, cudaMemcpyHostToDevice, st));
  GBI_CHECK(cudaMemcpyAsync(ctx->hVa.p, Va, v3, cudaMemcpyHostToDevice, st));
  GBI_CHECK(cudaMemcpyAsync(ctx->hOa.p, Oa, v3, cudaMemcpyHostToDevice, st));
  GBI_CHECK(cudaMemcpyAsync(ctx->hVH.p, VH, vh, cudaMemcpyHostToDevice, st));
  GBI_CHECK(cudaMemcpyAsync(ctx->hFe.p, Fe, v3, cudaMemcpyHostToDevice, st));
  GBI_CHECK(cudaMemcpyAsync(ctx->hTe.p, Te, v3, cudaMemcpyHostToDevice, st));
  if (warm_start) GBI_CHECK(cudaMemcpyAsync(ctx->hQH.p, QH, vh, cudaMemcpyHostToDevice, st));
  gbi_status s = gbi_solve(ctx, prm, N, P<double>(ctx->hR), P<double>(ctx->hVa), P<double>(ctx->hOa),
                           P<double>(ctx->hVH), P<double>(ctx->hFe), P<double>(ctx->hTe), P<double>(ctx->hV),
                           P<double>(ctx->hOm), P<double>(ctx->hQH), warm_start, info);
  if (s != GBI_OK && s != GBI_ERR_NOT_CONVERGED) return s;
  GBI_CHECK(cudaMemcpyAsync(V, ctx->hV.p, v3, cudaMemcpyDeviceToHost, st));
  GBI_CHECK(cudaMemcpyAsync(Omega, ctx->hOm.p, v3, cudaMemcpyDeviceToHost, st));
  if (QH) GBI_CHECK(cudaMemcpyAsync(QH, ctx->hQH.p, vh, cudaMemcpyDeviceToHost, st));
  GBI_CHECK(cudaStreamSynchronize(st));
  return s;
}

}  // extern "C"

// =================================================================================
// Solve without allocation: the whole workspace lives in one file-scope device array.
// =================================================================================

namespace {

constexpr int kStaticMaxN = 1024;         // spheres
constexpr int kStaticMaxNH = 8192;        // spheres x higher components (N * gbi_h(trunc))
constexpr int kStaticMaxRestart = 32;     // Krylov vectors per GMRES cycle
constexpr int kStaticMaxND = kStaticMaxNH + 6 * kStaticMaxN;

constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of every workspace buffer gbi_solve touches
constexpr size_t kOffHi = 0;
constexpr size_t kOffLo = kOffHi + al256(sizeof(float) * 4 * kStaticMaxN);
constexpr size_t kOff64 = kOffLo + al256(sizeof(float) * 4 * kStaticMaxN);
constexpr size_t kOffXQ = kOff64 + al256(sizeof(double) * 4 * kStaticMaxN);
constexpr size_t kOffXVH = kOffXQ + al256(sizeof(double) * kStaticMaxND);
constexpr size_t kOffB = kOffXVH + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffR = kOffB + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffDelta = kOffR + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffXVL = kOffDelta + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffKry = kOffXVL + al256(sizeof(double) * 6 * kStaticMaxN);
constexpr size_t kOffW = kOffKry + al256(sizeof(double) * (size_t)(kStaticMaxRestart + 1) * kStaticMaxNH);
constexpr size_t kOffPart = kOffW + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffDots = kOffPart + al256(sizeof(double) * 64 * (kMaxRestart + 2));
constexpr size_t kOffMin = kOffDots + al256(sizeof(double) * (2 * kMaxRestart + 8));
constexpr size_t kOffX32 = kOffMin + 256;
constexpr size_t kOffGs = kOffX32 + al256(sizeof(float) * 2 * (kStaticMaxND + 3 * kStaticMaxN));
constexpr size_t kOffBoff = kOffGs + al256(sizeof(double) * (64 + (kStaticMaxRestart + 1) * kStaticMaxRestart +
                                                              8 * (kStaticMaxRestart + 1) +
                                                              48 * (2 * (kStaticMaxRestart + 1) + 1) +
                                                              kFusedBlocks * (2 * (kStaticMaxRestart + 1) + 1) + 24));
constexpr size_t kOffBsys = kOffBoff + 256;
constexpr size_t kStaticBytes = kOffBsys + al256(sizeof(int) * kStaticMaxN);

// The scratch itself (about 2.6 MB).  Every device that loads the library holds it
// until the process exits.  Host code must not use this symbol as an address.
__device__ __align__(256) unsigned char g_solve_scratch[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
void* g_scratch_addr[kStaticMaxDevices] = {nullptr};   // device address, per device ordinal
double g_static_scalars[2 * kMaxRestart + 16];          // host read-back scalars (pageable)

}  // namespace

extern "C" gbi_status gbi_solve_static(void* stream, const gbi_params* prm, int N, const double* R,
                                       const double* Va, const double* Oa, const double* VH, const double* Fe,
                                       const double* Te, double* V, double* Omega, double* QH, int warm_start,
                                       gbi_info* info) {
  if (!valid_params(prm) || N < 0) return GBI_ERR_ARG;
  const int h = gbi_h(prm->trunc);
  if (N > kStaticMaxN || (long long)N * h > kStaticMaxNH) return GBI_ERR_ARG;
  if (prm->restart > kStaticMaxRestart) return GBI_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return GBI_ERR_CUDA;
  if (g_scratch_addr[dev] == nullptr) {
    // one-time set-up on this device: the device address of the static array
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_solve_scratch) != cudaSuccess || p == nullptr) return GBI_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  gbi_ctx c;
  c.device = dev;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  c.hbuf = g_static_scalars;
  c.allow_graphs = false;      // graph instantiation could allocate
  c.fixed = true;
  auto bind = [&](Buf& b, size_t off, size_t bytes) {
    b.p = base + off;
    b.bytes = bytes;
  };
  bind(c.pos_hi, kOffHi, kOffLo - kOffHi);
  bind(c.pos_lo, kOffLo, kOff64 - kOffLo);
  bind(c.pos64, kOff64, kOffXQ - kOff64);
  bind(c.xQ, kOffXQ, kOffXVH - kOffXQ);
  bind(c.xVH, kOffXVH, kOffB - kOffXVH);
  bind(c.b, kOffB, kOffR - kOffB);
  bind(c.r, kOffR, kOffDelta - kOffR);
  bind(c.delta, kOffDelta, kOffXVL - kOffDelta);
  bind(c.xVL, kOffXVL, kOffKry - kOffXVL);
  bind(c.krylov, kOffKry, kOffW - kOffKry);
  bind(c.w, kOffW, kOffPart - kOffW);
  bind(c.partial, kOffPart, kOffDots - kOffPart);
  bind(c.dots, kOffDots, kOffMin - kOffDots);
  bind(c.minr2, kOffMin, 256);
  bind(c.x32, kOffX32, kOffGs - kOffX32);
  bind(c.gstate, kOffGs, kOffBoff - kOffGs);
  bind(c.boff, kOffBoff, 256);
  bind(c.bsys, kOffBsys, kStaticBytes - kOffBsys);
  gbi_params p = *prm;
  if (p.restart <= 0) p.restart = kStaticMaxRestart;
  return gbi_solve(&c, &p, N, R, Va, Oa, VH, Fe, Te, V, Omega, QH, warm_start, info);
}
