// Shared parts of libgbi: pair-pass dispatch and bookkeeping, workspace management,
// input packing kernels, per-call set-up and batch layouts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "pair_chunk.cuh"
#include "pair_tile.cuh"

namespace gbi {
#define GBI_DECL(P)                                                                       \
  cudaError_t launch_pairs_##P##_2(int, int, const PairArgs&, cudaStream_t);              \
  cudaError_t launch_pairs_##P##_3(int, int, const PairArgs&, cudaStream_t);              \
  cudaError_t launch_pairs_##P##_4(int, int, const PairArgs&, cudaStream_t);
GBI_DECL(f32)
GBI_DECL(f64)
GBI_DECL(df)
#undef GBI_DECL
cudaError_t launch_pairs_f64_5(int, int, const PairArgs&, cudaStream_t);
cudaError_t launch_pairs_f64_40(int, int, const PairArgs&, cudaStream_t);

// precision: 0 = FP64, 1 = FP32, 2 = double-float on the FP32 pipe
cudaError_t launch_pairs(int trunc, int rows, int cols, int precision, const PairArgs& args,
                         cudaStream_t stream) {
#define GBI_DISPATCH(P)                                                   \
  if (trunc == 2) return launch_pairs_##P##_2(rows, cols, args, stream);  \
  if (trunc == 3) return launch_pairs_##P##_3(rows, cols, args, stream);  \
  if (trunc == 4) return launch_pairs_##P##_4(rows, cols, args, stream);  \
  return cudaErrorInvalidValue;
  // l <= 5 and the minimal set: FP64 passes only
  if (fp64_only(trunc)) {
    if (precision != 0) return cudaErrorInvalidValue;
    return trunc == 5 ? launch_pairs_f64_5(rows, cols, args, stream) : launch_pairs_f64_40(rows, cols, args, stream);
  }
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
  if (trunc == 5) return gbi_t5_flops[rows][cols];
  if (trunc == 40) return gbi_t40_flops[rows][cols];
  return 0.0;
}
}  // namespace gbi

namespace gbi {

gbi_status fail(gbi_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return GBI_OK;
  // the allocation-free entry point keeps no message (it has no handle to read it from)
  if (!c->fixed) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? GBI_ERR_NOMEM : GBI_ERR_CUDA;
}

gbi_status host_scratch(gbi_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->hs_cap) return GBI_OK;
  if (ctx->fixed) return GBI_ERR_NOMEM;   // static storage: never reallocated
  ctx->hs_own.resize(bytes);
  ctx->hs = ctx->hs_own.data();
  ctx->hs_cap = bytes;
  return GBI_OK;
}

gbi_status ensure(gbi_ctx* ctx, Buf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return GBI_OK;
  if (ctx->fixed) return GBI_ERR_NOMEM;   // static storage: never reallocated
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
  const int D = d_of(trunc);
  return cols == SET_L ? 6 : cols == SET_H ? D - 6 : D;
}

gbi_status status_words(gbi_ctx* ctx) {
  const void* old = ctx->minr2.p;
  GBI_TRY(ensure(ctx, ctx->minr2, 4 * sizeof(unsigned int)));
  if (ctx->minr2.p != old) GBI_CHECK(cudaMemsetAsync(ctx->minr2.p, 0, 4 * sizeof(unsigned int), ctx->stream));
  return GBI_OK;
}

int* pass_error_word(gbi_ctx* ctx) { return P<int>(ctx->minr2) + 1; }
int* input_error_word(gbi_ctx* ctx) { return P<int>(ctx->minr2) + 2; }

gbi_status tile_reserve(gbi_ctx* ctx, int trunc, int rows, int precision, int N, TilePlan* out) {
  const TilePlan t = tile_plan(N, sm_count(ctx), 1);
  if (t.P <= 0) return GBI_ERR_ARG;
  const int D = d_of(trunc);
  const int nr = rows == SET_L ? 6 : (rows == SET_H ? D - 6 : D);
  GBI_TRY(ensure(ctx, ctx->tile, tile_part_bytes(t, nr, precision == 2 ? sizeof(df) : sizeof(float))));
  const void* old = ctx->tilecnt.p;
  GBI_TRY(ensure(ctx, ctx->tilecnt, sizeof(unsigned int) * (size_t)t.G));
  // counters start at zero and every launch leaves them so; a new buffer is cleared
  if (ctx->tilecnt.p != old) GBI_CHECK(cudaMemsetAsync(ctx->tilecnt.p, 0, ctx->tilecnt.bytes, ctx->stream));
  GBI_TRY(status_words(ctx));
  if (out) *out = t;
  return GBI_OK;
}

gbi_status pass_error_reset(gbi_ctx* ctx) {
  GBI_CHECK(cudaMemsetAsync(pass_error_word(ctx), 0, sizeof(int), ctx->stream));
  if (ctx->tilecnt.p) GBI_CHECK(cudaMemsetAsync(ctx->tilecnt.p, 0, ctx->tilecnt.bytes, ctx->stream));
  return GBI_OK;
}

gbi_status chunk_reserve(gbi_ctx* ctx, int trunc, int rows, int precision, int N, ChunkPlan* out) {
  const ChunkPlan c = chunk_plan(N, sm_count(ctx), chunk_warps_sm(trunc, precision));
  if (c.P <= 0) return GBI_ERR_ARG;
  const int D = d_of(trunc);
  const int nr = rows == SET_L ? 6 : (rows == SET_H ? D - 6 : D);
  GBI_TRY(ensure(ctx, ctx->tile, chunk_part_bytes(c, N, nr, precision == 2 ? sizeof(df) : sizeof(float))));
  const void* old = ctx->tilecnt.p;
  GBI_TRY(ensure(ctx, ctx->tilecnt, sizeof(unsigned int) * (size_t)N));
  // counters start at zero and every launch leaves them so; a new buffer is cleared
  if (ctx->tilecnt.p != old) GBI_CHECK(cudaMemsetAsync(ctx->tilecnt.p, 0, ctx->tilecnt.bytes, ctx->stream));
  GBI_TRY(status_words(ctx));
  if (out) *out = c;
  return GBI_OK;
}

bool balanced_args(gbi_ctx* ctx, int trunc, int rows, int precision, int N, PairArgs& a) {
  if (a.wpt == kFormTile) {
    TilePlan t;
    if (tile_reserve(ctx, trunc, rows, precision, N, &t) != GBI_OK) return false;
    a.tile_P = t.P;
    a.tile_G = t.G;
    a.tile_maxseg = t.maxseg;
  } else {
    ChunkPlan c;
    if (chunk_reserve(ctx, trunc, rows, precision, N, &c) != GBI_OK) return false;
    a.tile_P = c.P;
    a.tile_G = c.G;
    a.tile_maxseg = c.maxseg;
  }
  a.tile_part = ctx->tile.p;
  a.tile_cnt = P<unsigned int>(ctx->tilecnt);
  a.err = pass_error_word(ctx);
  a.wait_limit = ctx->wait_limit;
  return true;
}

// A balanced form (tiled or chunk-balanced) for this pass if the caller's (or the tuned)
// choice asks for it and its scratch can be had (a context bound to static storage may
// not have it): fills the plan and scratch fields of a; otherwise a's wpt is set back to
// a streaming choice.
void tile_select(gbi_ctx* ctx, int trunc, int rows, int precision, PairArgs& a) {
  const bool batched = a.sys_of != nullptr && a.nsys > 1;
  if (precision == 0 || !balanced_form(a.wpt) || batched || a.N <= 1) {
    if (balanced_form(a.wpt)) a.wpt = 0;
    return;
  }
  if (!balanced_args(ctx, trunc, rows, precision, a.N, a)) a.wpt = 0;
}

// Split of the streaming form's last, partly filled wave (see PairArgs::split_from): with
// `slots` resident blocks, N = full * slots + r targets take full + 1 waves of whole-target
// blocks; split into ns parts, the last r targets take ceil(r ns / slots) waves of 1/ns of a
// block instead.  ns (2..8) minimises that, charging 2% of a block per part for the extra
// reductions and stores; no split unless it saves more than that.
void split_plan(int N, int slots, int& split_from, int& nsplit) {
  split_from = 0x7fffffff;
  nsplit = 1;
  if (slots <= 0 || N <= slots || N % slots == 0) return;
  const int r = N % slots, full = N / slots;
  double best = full + 1.0;
  for (int ns = 2; ns <= 8; ++ns) {
    const double c = full + double((r * ns + slots - 1) / slots) / ns + 0.02 * ns;
    if (c < best - 1e-9) {
      best = c;
      nsplit = ns;
    }
  }
  if (nsplit > 1) split_from = N - r;
}

// the split's scratch: one row block per part of each split target, one arrival counter
// per split target (zero between launches; a new buffer is cleared)
bool split_reserve(gbi_ctx* ctx, int trunc, int rows, int precision, PairArgs& a) {
  const int wpt = stream_wpt(trunc, precision, a.N, a.wpt);
  const int warps_sm = (trunc == 4 || precision == 2) ? 8 : 16;
  int from = 0, ns = 1;
  split_plan(a.N, sm_count(ctx) * std::max(1, warps_sm / wpt), from, ns);
  if (ns <= 1) return false;
  const int D = d_of(trunc);
  const int nr = rows == SET_L ? 6 : (rows == SET_H ? D - 6 : (rows == SET_P ? 3 : D));
  const size_t nrc32 = (size_t)((nr + 31) / 32) * 32;
  const int tail = a.N - from;
  if (ensure(ctx, ctx->tile, sizeof(double) * (size_t)tail * ns * nrc32) != GBI_OK) return false;
  const void* old = ctx->tilecnt.p;
  if (ensure(ctx, ctx->tilecnt, sizeof(unsigned int) * (size_t)a.N) != GBI_OK) return false;
  if (ctx->tilecnt.p != old && cudaMemsetAsync(ctx->tilecnt.p, 0, ctx->tilecnt.bytes, ctx->stream) != cudaSuccess)
    return false;
  a.tile_part = ctx->tile.p;
  a.tile_cnt = P<unsigned int>(ctx->tilecnt);
  a.split_from = from;
  a.nsplit = ns;
  return true;
}

cudaError_t run_pairs(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, const PairArgs& args_in) {
  const double pairs = args_in.npairs > 0 ? double(args_in.npairs) : double(args_in.N) * double(args_in.N - 1);
  const double flops = pair_flops(trunc, rows, cols) * pairs;
  PairArgs args = args_in;
  int extra = 0;
  if (args.wpt == 0)
    args.wpt = ctx->force_wpt > 0 ? ctx->force_wpt
                                  : ctx->tuned_wpt(trunc, rows, cols, precision, args.N,
                                                   args.sys_of != nullptr && args.nsys > 1);
  tile_select(ctx, trunc, rows, precision, args);
  if (precision >= 1 && !balanced_form(args.wpt) && !(args.sys_of != nullptr && args.nsys > 1) &&
      ctx->split_tail)
    split_reserve(ctx, trunc, rows, precision, args);
  if (precision == 2 || (precision == 1 && args.x32 == nullptr)) {
    // per-sphere source records (FP32, or the double-float hi/lo pair), once per pass,
    // so that the pair loop touches no FP64
    const int nc = ncols_of(trunc, cols);
    const size_t bytes = sizeof(float) * rec_floats(nc, precision == 2) * (size_t)args.N;
    if (ensure(ctx, ctx->x32, bytes) != GBI_OK) return cudaErrorMemoryAllocation;
    ColScale cs;
    const int c0 = cols == SET_H ? 6 : 0;
    for (int i = 0; i < kMaxD; ++i) cs.v[i] = (i < nc) ? args.colscale[c0 + i] : 1.0;
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

int d_of(int trunc) {
  switch (trunc) {
    case 2: return GbiTrunc2::D;
    case 3: return GbiTrunc3::D;
    case 4: return GbiTrunc4::D;
    case 5: return GbiTrunc5::D;
    case 40: return GbiTrunc40::D;
    default: return -1;
  }
}
const double* scale_tab(int trunc) {
  switch (trunc) {
    case 2: return gbi_t2_scale;
    case 3: return gbi_t3_scale;
    case 4: return gbi_t4_scale;
    case 5: return gbi_t5_scale;
    default: return gbi_t40_scale;
  }
}
const double* self_tab(int trunc) {
  switch (trunc) {
    case 2: return gbi_t2_self;
    case 3: return gbi_t3_self;
    case 4: return gbi_t4_self;
    case 5: return gbi_t5_self;
    default: return gbi_t40_self;
  }
}

// ---------------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------------

// non-finite inputs: any NaN or infinity among v0..v2 sets *bad (if given)
__device__ __forceinline__ void flag_nonfinite(int* bad, double v0, double v1, double v2) {
  if (bad != nullptr && !(isfinite(v0) && isfinite(v1) && isfinite(v2))) atomicOr(bad, 1);
}

__global__ void k_positions(int N, const double* __restrict__ R, float4* hi, float4* lo, dpos4* p64, int* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double x = R[3 * n], y = R[3 * n + 1], z = R[3 * n + 2];
  flag_nonfinite(bad, x, y, z);
  const float hx = float(x), hy = float(y), hz = float(z);
  hi[n] = make_float4(hx, hy, hz, 0.f);
  lo[n] = make_float4(float(x - double(hx)), float(y - double(hy)), float(z - double(hz)), 0.f);
  p64[n] = dpos4{x, y, z, 0.0};
}

// F^(1) = -F^e and F^(21) = -T^e/a in internal coordinates: xF[6][N]
__global__ void k_pack_lower(int N, double a, double c2a, const double* __restrict__ Fe,
                             const double* __restrict__ Te, double* xF, int* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double* f = Fe + 3 * n;
  const double* t = Te + 3 * n;
  flag_nonfinite(bad, f[0], f[1], f[2]);
  flag_nonfinite(bad, t[0], t[1], t[2]);
  xF[0 * N + n] = -f[1];
  xF[1 * N + n] = -f[2];
  xF[2 * N + n] = -f[0];
  xF[3 * N + n] = -c2a * t[1] / a;
  xF[4 * N + n] = -c2a * t[2] / a;
  xF[5 * N + n] = -c2a * t[0] / a;
}

// packed [N][h] -> internal component-major [h][N] times scale * mult
__global__ void k_pack_higher(int N, int h, const double* __restrict__ VH, Scales sc, double mult,
                              double* out, int* bad) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= (size_t)N * h) return;
  const int n = int(i / h), p = int(i - (size_t)n * h);
  flag_nonfinite(bad, VH[i], 0.0, 0.0);
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
                                 double* V, double* Om, int* bad) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  flag_nonfinite(bad, Va[3 * n], Va[3 * n + 1], Va[3 * n + 2]);
  flag_nonfinite(bad, Oa[3 * n], Oa[3 * n + 1], Oa[3 * n + 2]);
  const double f = 1.0 / (c2a * 2.0 * a);
  V[3 * n + 0] = Va[3 * n + 0] + xVL[2 * N + n];
  V[3 * n + 1] = Va[3 * n + 1] + xVL[0 * N + n];
  V[3 * n + 2] = Va[3 * n + 2] + xVL[1 * N + n];
  Om[3 * n + 0] = Oa[3 * n + 0] + f * xVL[5 * N + n];
  Om[3 * n + 1] = Oa[3 * n + 1] + f * xVL[3 * N + n];
  Om[3 * n + 2] = Oa[3 * n + 2] + f * xVL[4 * N + n];
}

// ---------------------------------------------------------------------------------
// solver state for one call
// ---------------------------------------------------------------------------------

gbi_status setup_call(gbi_ctx* ctx, Setup& s, int N, int trunc, double a, double eta, const double* R,
                      bool launch) {
  s.N = N;
  s.trunc = trunc;
  s.D = d_of(trunc);
  s.h = s.D - 6;
  s.a = a;
  s.eta = eta;
  const double* sc = scale_tab(trunc);
  const double* sg = self_tab(trunc);
  for (int i = 0; i < kMaxD; ++i) {
    s.scale.v[i] = i < s.D ? sc[i] : 1.0;
    s.selfg.v[i] = i < s.D ? sg[i] : 0.0;
    s.ones.v[i] = 1.0;
    s.minv.v[i] = (i < s.h) ? a / sg[6 + i] : 1.0;
  }
  s.pairs_per_pass = (long long)N * (N - 1);
  GBI_TRY(ensure(ctx, ctx->pos_hi, sizeof(float4) * N));
  GBI_TRY(ensure(ctx, ctx->pos_lo, sizeof(float4) * N));
  GBI_TRY(ensure(ctx, ctx->pos64, sizeof(dpos4) * N));
  s.pos = Positions{P<float4>(ctx->pos_hi), P<float4>(ctx->pos_lo), P<dpos4>(ctx->pos64)};
  if (launch) GBI_TRY(launch_positions(ctx, s, R));
  return GBI_OK;
}

gbi_status launch_positions(gbi_ctx* ctx, const Setup& s, const double* R, int* bad) {
  k_positions<<<grid1(s.N), 256, 0, ctx->stream>>>(s.N, R, P<float4>(ctx->pos_hi), P<float4>(ctx->pos_lo),
                                                   P<dpos4>(ctx->pos64), bad);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
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
  p.wpt = 0;
  p.y = y;
  p.alpha = alpha;
  p.beta = beta;
  p.add_self = add_self;
  for (int i = 0; i < kMaxD; ++i) {
    // colscale is indexed by absolute component; callers pass H-relative scales with col0 = 6
    const int src = i - col0;
    p.colscale[i] = (src >= 0 && src < kMaxD) ? colscale.v[src] : 1.0;
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
  p.nsys = 1;
  p.npairs = 0;
  p.pdl = 0;
  p.tile_part = nullptr;
  p.tile_cnt = nullptr;
  p.tile_P = p.tile_G = p.tile_maxseg = 0;
  p.err = nullptr;
  p.wait_limit = 0;
  p.split_from = 0x7fffffff;
  p.nsplit = 1;
  return p;
}

// streaming multiprocessors of the context's device (cached)
int sm_count(gbi_ctx* ctx) {
  if (ctx->num_sms == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || v <= 0) v = 152;
    ctx->num_sms = v;
  }
  return ctx->num_sms;
}

// S = 1 batch over the spheres [0, N): offsets and system ids in the context workspace
gbi_status single_batch(gbi_ctx* ctx, int N, Batch& B) {
  GBI_TRY(ensure(ctx, ctx->boff, sizeof(int) * 2));
  GBI_TRY(ensure(ctx, ctx->bsys, sizeof(int) * (size_t)std::max(N, 1)));
  // the arrays already describe one system of N spheres unless a batch call or a
  // reallocation changed them since
  if (ctx->single_N != N || ctx->single_off != ctx->boff.p || ctx->single_sys != ctx->bsys.p) {
    ctx->single_N = N;
    ctx->single_off = ctx->boff.p;
    ctx->single_sys = ctx->bsys.p;
    ctx->single_off_host[0] = 0;
    ctx->single_off_host[1] = N;
    GBI_CHECK(cudaMemcpyAsync(ctx->boff.p, ctx->single_off_host, sizeof(int) * 2, cudaMemcpyHostToDevice,
                              ctx->stream));
    GBI_CHECK(cudaMemsetAsync(ctx->bsys.p, 0, sizeof(int) * (size_t)N, ctx->stream));
  }
  B.S = 1;
  B.Ntot = N;
  B.off = P<int>(ctx->boff);
  B.sys = P<int>(ctx->bsys);
  B.one[0] = 0;
  B.one[1] = N;
  B.h_off = B.one;
  return GBI_OK;
}

__global__ void k_fill_sys(int S, const int* __restrict__ off, int* sys) {
  const int s = blockIdx.x;
  for (int p = off[s] + threadIdx.x; p < off[s + 1]; p += blockDim.x) sys[p] = s;
}

long long batch_pairs(const Batch& B) {
  long long c = 0;
  for (int q = 0; q < B.S; ++q) {
    const long long n = B.h_off[q + 1] - B.h_off[q];
    c += n * (n - 1);
  }
  return c;
}

bool valid_offsets(int nsys, const int* off) {
  if (off[0] != 0) return false;
  for (int q = 0; q < nsys; ++q)
    if (off[q + 1] < off[q]) return false;
  return true;
}

// Device copies of a batch layout (system offsets and the system of every sphere).
gbi_status make_batch(gbi_ctx* ctx, int nsys, const int* offsets_host, Batch& B) {
  ctx->single_N = -1;   // the batch arrays are rewritten below
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
  B.h_off = offsets_host;
  return GBI_OK;
}

bool valid_params(const gbi_params* p) {
  if (!p) return false;
  if (!(p->a > 0) || !(p->eta > 0)) return false;
  if (d_of(p->trunc) < 0) return false;
  if (p->precision < 0 || p->precision > 3) return false;
  if (fp64_only(p->trunc) && p->precision != 0) return false;
  return true;
}

}  // namespace gbi
