// C ABI of libgbi: context, pair operator, solves, superposition, the harmonic-trap
// integrator, pair-kernel tuning, instrumentation and the allocation-free solve.
// Every arithmetic step of the method runs in the kernels of this library; the host
// only sequences launches and reads small per-system solver states back.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"
#include "gstate.cuh"
#include "pair_tile.cuh"

namespace gbi {
namespace {

__global__ void k_trap_inputs(int N, double k_trap, double vs, double s0, double d0, double q0, int h,
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
  // V^(4t) = q0 (pp - I/3): the degenerate octupole of a squirmer (trunc >= 3)
  if (h >= 25 && q0 != 0.0)
    for (int i = 0; i < 5; ++i) vh[20 + i] = q0 * q[i];
}

// One-body flow coefficients of the higher modes (Sec. IV: an isolated sphere's traction
// from its own active velocity, the self elements alone): Q^H = -8 pi eta a V^H / g, g the
// self scalars of a unit sphere.  [N][h] in and out.
__global__ void k_qh_onebody(int N, int h, const double* __restrict__ VH, Scales ginv, double mult,
                             double* __restrict__ QH) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)N * h) return;
  QH[i] = mult * VH[i] * ginv.v[i % h];
}

// Modes of a squirmer with the Lighthill-Blake slip of Sec. V, B1 and B2: from the slip's
// tensorial-harmonic coefficients, V^a = 2 B1 p / 3, V^(2s) = -3/5 B2 (pp - I/3),
// V^(3t) = 10/3 B1 p and V^(4t) = 7 B2 (pp - I/3) (the trap parameters vs, s0, d0, q0).
struct SquirmerModes {
  double vs, s0, d0, q0;
};
inline SquirmerModes squirmer_modes(double B1, double B2) {
  return SquirmerModes{2.0 * B1 / 3.0, -0.6 * B2, 10.0 * B1 / 3.0, 7.0 * B2};
}

// With rec set (a trap step replayed inside the solve graph) the update is skipped when
// that solve failed: an overlap, or a residual above rtol -- the cases in which the
// host-driven step stops before its update.
__global__ void k_euler(int N, double dt, const double* __restrict__ V, const double* __restrict__ Om,
                        double* R, double* p, const DSolve* __restrict__ rec = nullptr, double rtol = 0.0) {
  if (rec != nullptr && (rec->overlap || !(rec->rel_max <= rtol))) return;
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

constexpr int kTunedPasses = 6;

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
  // the FP32 and double-float passes of the mixed-precision solves (the right-hand-side
  // and output passes run in FP32 for precision 3, in double-float for precision 2)
  const Pass passes[kTunedPasses] = {{SET_H, SET_H, 1}, {SET_H, SET_H, 2}, {SET_H, SET_L, 2},
                                     {SET_L, SET_ALL, 2}, {SET_H, SET_L, 1}, {SET_L, SET_ALL, 1}};
  gbi_status st = GBI_OK;
  for (int k = 0; k < kTunedPasses && st == GBI_OK; ++k) {
    const Pass& ps = passes[k];
    PairArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.N = Ntot;
    pa.a = 1.0;
    pa.pos = Positions{hi, lo, nullptr};
    pa.x = x;
    pa.y = y;
    pa.alpha = 1.0;
    for (int i = 0; i < kMaxD; ++i) pa.colscale[i] = 1.0;
    if (batched) {
      pa.sys_of = sys_of;
      pa.sys_off = sys_off;
      pa.nsys = nsys;
    }
    const int nc = ncols_of(trunc, ps.cols);
    ColScale cs;
    for (int i = 0; i < kMaxD; ++i) cs.v[i] = 1.0;
    cudaError_t e = launch_records(ps.precision == 2, Ntot, nc, x, nullptr, 0, nullptr, cs, rec, ctx->stream);
    pa.x32 = rec;
    int best = 0;
    float best_ms = 0.f;
    // candidates: the tiled form (1, one system only) and 2, 4, ... warps per target of
    // the streaming form
    std::vector<int> cand;
    if (!batched) {
      cand.push_back(kFormTile);
      cand.push_back(kFormChunk);
    }
    for (int w = 2; w <= max_wpt(trunc, ps.precision); w *= 2) cand.push_back(w);
    for (const int w : cand) {
      if (e != cudaSuccess) break;
      pa.wpt = w;
      pa.nsplit = 0;
      if (balanced_form(w) && !balanced_args(ctx, trunc, ps.rows, ps.precision, Ntot, pa)) continue;
      if (!balanced_form(w) && !batched && ctx->split_tail) split_reserve(ctx, trunc, ps.rows, ps.precision, pa);
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
    ++ctx->wpt_gen;
    if (chosen) chosen[k] = best;
  }
  ctx->pool.push_back(e0);
  ctx->pool.push_back(e1);
  return st;
}

}  // namespace
}  // namespace gbi

using namespace gbi;

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
  *out = c;
  return GBI_OK;
}

gbi_status gbi_destroy(gbi_ctx* ctx) {
  if (!ctx) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  Buf* bufs[] = {&ctx->pos_hi, &ctx->pos_lo, &ctx->pos64, &ctx->b, &ctx->xQ, &ctx->r,
                 &ctx->delta, &ctx->krylov, &ctx->w, &ctx->xVL, &ctx->minr2, &ctx->x32, &ctx->trapbuf, &ctx->gstate, &ctx->boff, &ctx->bsys, &ctx->tFe, &ctx->tTe, &ctx->tVa, &ctx->tOa, &ctx->tVH, &ctx->tV, &ctx->tOm,
                 &ctx->tQH, &ctx->hR, &ctx->hVa, &ctx->hOa, &ctx->hVH, &ctx->hFe, &ctx->hTe, &ctx->hV,
                 &ctx->hOm, &ctx->hQH, &ctx->mlp_th, &ctx->mlp_m, &ctx->mlp_v, &ctx->mlp_thq, &ctx->mlp_pk,
                 &ctx->mlp_grad, &ctx->mlp_pk_tc, &ctx->mlp_err, &ctx->nb_cnt, &ctx->nb_start, &ctx->nb_tg, &ctx->nb_sr, &ctx->nb_scan,
                 &ctx->cell_of, &ctx->cell_cnt, &ctx->cell_start, &ctx->cell_fill, &ctx->cell_items, &ctx->nb_aux,
                 &ctx->mf_F, &ctx->mf_FR, &ctx->mf_lab, &ctx->mf_dO, &ctx->mf_part, &ctx->mf_loss, &ctx->dsolve,
                 &ctx->tile, &ctx->tilecnt, &ctx->flowx, &ctx->flowrec, &ctx->flowcnt, &ctx->wallbuf, &ctx->perbuf};
  for (Buf* b : bufs)
    if (b->p) cudaFree(b->p);
  drain_profile(ctx);
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  if (ctx->chunk_exec) cudaGraphExecDestroy(ctx->chunk_exec);
  if (ctx->solve_exec) cudaGraphExecDestroy(ctx->solve_exec);
  for (cudaStream_t cs : ctx->cap)
    if (cs) cudaStreamDestroy(cs);
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
  if (fp64_only(trunc) && precision != 0) return GBI_ERR_ARG;
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
  for (int i = 0; i < kMaxD; ++i) oneb.v[i] = (i < h) ? s.scale.v[6 + i] * s.a / s.selfg.v[6 + i] : 1.0;
  k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], Fe, Te, xF, nullptr);
  ++ctx->launches;
  k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, oneb, -8.0 * kPi * s.eta, xQH, nullptr);
  ++ctx->launches;
  PairArgs p = pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1, s.ones,
                         0);
  p.sys_of = B.sys;
  p.sys_off = B.off;
  p.nsys = B.S;
  p.npairs = batch_pairs(B);
  GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, prm->precision == 3 ? 1 : prm->precision, p));
  k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], P<double>(ctx->xVL), Va, Oa, V,
                                                      Omega, nullptr);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_qh_onebody(gbi_ctx* ctx, const gbi_params* prm, int N, const double* VH, double* QH) {
  if (!ctx || !valid_params(prm) || N < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!VH || !QH) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  const int h = gbi_h(prm->trunc);
  const double* sg = self_tab(prm->trunc);
  Scales ginv;   // 1 / g of every higher component (self scalars of a unit sphere)
  for (int i = 0; i < kMaxD; ++i) ginv.v[i] = i < h ? 1.0 / sg[6 + i] : 0.0;
  k_qh_onebody<<<grid1((size_t)N * h), 256, 0, ctx->stream>>>(N, h, VH, ginv, -8.0 * kPi * prm->eta * prm->a, QH);
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
  for (int i = 0; i < kMaxD; ++i) oneb.v[i] = (i < h) ? s.scale.v[6 + i] * s.a / s.selfg.v[6 + i] : 1.0;
  k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], Fe, Te, xF, nullptr);
  ++ctx->launches;
  k_pack_higher<<<grid1(nh), 256, 0, ctx->stream>>>(N, h, VH, oneb, -8.0 * kPi * s.eta, xQH, nullptr);
  ++ctx->launches;
  PairArgs p = pair_args(s, P<double>(ctx->xQ), P<double>(ctx->xVL), -1.0 / (8.0 * kPi * s.eta), 0.0, 1, s.ones,
                         0);
  GBI_CHECK(run_pairs(ctx, s.trunc, SET_L, SET_ALL, prm->precision == 3 ? 1 : prm->precision, p));
  k_finalize_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], P<double>(ctx->xVL), Va, Oa, V,
                                                      Omega, nullptr);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

}  // extern "C"

namespace gbi {
namespace {

// Forward-Euler trap steps of one suspension (nsys = 1, offsets NULL) or of a batch of
// independent ones (system s = spheres [offsets[s], offsets[s+1]), each with its own trap
// centred at the origin of the coordinates).
gbi_status trap_steps(gbi_ctx* ctx, const gbi_params* prm, int nsys, const int* offsets, int N, double dt,
                      double k_trap, double vs, double s0, double d0, double q0, int superposition, int nsteps,
                      double* R, double* p, gbi_info* info) {
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
  auto trap_inputs = [&]() -> gbi_status {
    k_trap_inputs<<<grid1(N), 256, 0, ctx->stream>>>(N, k_trap, vs, s0, d0, q0, h, R, p, P<double>(ctx->tFe),
                                                     P<double>(ctx->tTe), P<double>(ctx->tVa), P<double>(ctx->tOa),
                                                     P<double>(ctx->tVH));
    ++ctx->launches;
    GBI_CHECK(cudaGetLastError());
    return GBI_OK;
  };
  const double rtol = prm->rtol > 0 ? prm->rtol : 1e-10;
  auto euler = [&](const DSolve* rec) -> gbi_status {
    k_euler<<<grid1(N), 256, 0, ctx->stream>>>(N, dt, P<double>(ctx->tV), P<double>(ctx->tOm), R, p, rec, rtol);
    ++ctx->launches;
    GBI_CHECK(cudaGetLastError());
    return GBI_OK;
  };
  // the solve's work around it: inputs from (R, p) before, the update after (captured
  // with a replayed solve graph)
  StepHooks hooks;
  hooks.before = trap_inputs;
  hooks.after = euler;
  {
    double pr[6] = {dt, k_trap, vs, s0, d0, q0};
    long long b[6];
    std::memcpy(b, pr, sizeof(pr));
    hooks.key.assign(b, b + 6);
    hooks.key.push_back((long long)(uintptr_t)R);
    hooks.key.push_back((long long)(uintptr_t)p);
  }
  for (int step = 0; step < nsteps; ++step) {
    if (superposition) {
      GBI_TRY(trap_inputs());
      if (offsets == nullptr) {
        GBI_TRY(gbi_superpose(ctx, prm, N, R, P<double>(ctx->tVa), P<double>(ctx->tOa), P<double>(ctx->tVH),
                              P<double>(ctx->tFe), P<double>(ctx->tTe), P<double>(ctx->tV), P<double>(ctx->tOm)));
        total.pair_interactions += (long long)N * (N - 1);
      } else {
        GBI_TRY(gbi_batch_superpose(ctx, prm, nsys, offsets, R, P<double>(ctx->tVa), P<double>(ctx->tOa),
                                    P<double>(ctx->tVH), P<double>(ctx->tFe), P<double>(ctx->tTe), P<double>(ctx->tV),
                                    P<double>(ctx->tOm)));
        for (int q = 0; q < nsys; ++q) {
          const long long n = offsets[q + 1] - offsets[q];
          total.pair_interactions += n * (n - 1);
        }
      }
      (prm->precision == 1 || prm->precision == 3 ? total.matvecs_f32 : total.matvecs_f64) += 1;
      GBI_TRY(euler(nullptr));
    } else {
      gbi_info one{};
      // FP64 solves warm-start from the previous step's traction coefficients (also across
      // calls with the same N and truncation on this context).  Mixed-precision solves start
      // from zero: a warm start costs one more high-precision residual pass, and the FP32
      // inner solves cannot reach the target from it in fewer sweeps.
      const bool warm = prm->precision == 0 && (step > 0 || (ctx->tqh_N == N && ctx->tqh_trunc == prm->trunc));
      ctx->tqh_N = -1;
      Batch B;
      if (offsets == nullptr) GBI_TRY(single_batch(ctx, N, B));
      else GBI_TRY(make_batch(ctx, nsys, offsets, B));
      st = solve_core(ctx, prm, B, R, P<double>(ctx->tVa), P<double>(ctx->tOa), P<double>(ctx->tVH),
                      P<double>(ctx->tFe), P<double>(ctx->tTe), P<double>(ctx->tV), P<double>(ctx->tOm),
                      P<double>(ctx->tQH), warm ? 1 : 0, &one, &hooks);
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
      if (st != GBI_OK) break;   // the update ran only for a successful solve
    }
  }
  if (info) *info = total;
  return st;
}

}  // namespace
}  // namespace gbi

extern "C" {

gbi_status gbi_trap_step(gbi_ctx* ctx, const gbi_params* prm, int N, double dt, double k_trap, double vs,
                         double s0, double d0, int superposition, int nsteps, double* R, double* p,
                         gbi_info* info) {
  return trap_steps(ctx, prm, 1, nullptr, N, dt, k_trap, vs, s0, d0, 0.0, superposition, nsteps, R, p, info);
}

gbi_status gbi_squirmer_step(gbi_ctx* ctx, const gbi_params* prm, int N, double dt, double k_trap, double B1,
                             double B2, int superposition, int nsteps, double* R, double* p, gbi_info* info) {
  const SquirmerModes m = squirmer_modes(B1, B2);
  return trap_steps(ctx, prm, 1, nullptr, N, dt, k_trap, m.vs, m.s0, m.d0, m.q0, superposition, nsteps, R, p,
                    info);
}

gbi_status gbi_batch_trap_step(gbi_ctx* ctx, const gbi_params* prm, int nsys, const int* offsets_host, double dt,
                               double k_trap, double vs, double s0, double d0, int superposition, int nsteps,
                               double* R, double* p, gbi_info* info) {
  if (!ctx || nsys < 1 || !offsets_host || !valid_offsets(nsys, offsets_host)) return GBI_ERR_ARG;
  return trap_steps(ctx, prm, nsys, offsets_host, offsets_host[nsys], dt, k_trap, vs, s0, d0, 0.0, superposition,
                    nsteps, R, p, info);
}

gbi_status gbi_trap_inputs(gbi_ctx* ctx, int N, int trunc, double k_trap, double vs, double s0, double d0,
                           const double* R, const double* p, double* Fe, double* Te, double* Va, double* Oa,
                           double* VH) {
  if (!ctx || N < 0 || d_of(trunc) < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !p || !Fe || !Te || !Va || !Oa || !VH) return GBI_ERR_ARG;
  k_trap_inputs<<<grid1(N), 256, 0, ctx->stream>>>(N, k_trap, vs, s0, d0, 0.0, gbi_h(trunc), R, p, Fe, Te, Va, Oa,
                                                   VH);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_squirmer_inputs(gbi_ctx* ctx, int N, int trunc, double k_trap, double B1, double B2,
                               const double* R, const double* p, double* Fe, double* Te, double* Va, double* Oa,
                               double* VH) {
  if (!ctx || N < 0 || d_of(trunc) < 0) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !p || !Fe || !Te || !Va || !Oa || !VH) return GBI_ERR_ARG;
  const SquirmerModes m = squirmer_modes(B1, B2);
  k_trap_inputs<<<grid1(N), 256, 0, ctx->stream>>>(N, k_trap, m.vs, m.s0, m.d0, m.q0, gbi_h(trunc), R, p, Fe, Te,
                                                   Va, Oa, VH);
  ++ctx->launches;
  GBI_CHECK(cudaGetLastError());
  return GBI_OK;
}

gbi_status gbi_tune(gbi_ctx* ctx, int trunc, int nsys, const int* offsets, int reps, int* chosen) {
  if (!ctx || d_of(trunc) < 0 || fp64_only(trunc) || nsys < 1 || !offsets || reps < 0) return GBI_ERR_ARG;
  if (offsets[0] != 0) return GBI_ERR_ARG;
  for (int s = 0; s < nsys; ++s)
    if (offsets[s + 1] <= offsets[s]) return GBI_ERR_ARG;
  if (reps == 0) reps = 5;
  return tune_impl(ctx, trunc, nsys, offsets, reps, chosen);
}

gbi_status gbi_set_wpt(gbi_ctx* ctx, int wpt) {
  if (!ctx || !(wpt == 0 || wpt == 1 || wpt == 2 || wpt == 3 || wpt == 4 || wpt == 8 || wpt == 16)) return GBI_ERR_ARG;
  ctx->force_wpt = wpt;
  ++ctx->wpt_gen;
  return GBI_OK;
}

gbi_status gbi_set_split_tail(gbi_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return GBI_ERR_ARG;
  ctx->split_tail = on;
  ++ctx->wpt_gen;   // captured solve graphs hold the old launches
  return GBI_OK;
}

gbi_status gbi_set_wait_limit(gbi_ctx* ctx, long long rounds) {
  if (!ctx || rounds < -1) return GBI_ERR_ARG;
  ctx->wait_limit = rounds == -1 ? kTileWaitLimit : rounds;
  return GBI_OK;
}

gbi_status gbi_pass_status(gbi_ctx* ctx) {
  if (!ctx) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->minr2.p == nullptr) {
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    return GBI_OK;
  }
  int word = 0;
  GBI_CHECK(cudaMemcpyAsync(&word, pass_error_word(ctx), sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  if (word == 0) return GBI_OK;
  GBI_TRY(pass_error_reset(ctx));
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  return GBI_ERR_TIMEOUT;
}

int gbi_pass_wpt(gbi_ctx* ctx, int trunc, int rows, int cols, int precision, int N, int batched) {
  if (!ctx || d_of(trunc) < 0 || rows < 0 || rows > 2 || cols < 0 || cols > 2 || N < 1) return -1;
  if (precision == 0) return 0;
  if ((precision != 1 && precision != 2) || fp64_only(trunc)) return -1;
  const int req = ctx->force_wpt > 0 ? ctx->force_wpt : ctx->tuned_wpt(trunc, rows, cols, precision, N, batched != 0);
  return stream_wpt(trunc, precision, N, req, batched != 0);
}

gbi_status gbi_set_profiling(gbi_ctx* ctx, int on) {
  if (!ctx) return GBI_ERR_ARG;
  drain_profile(ctx);
  ctx->prof = on != 0;
  for (int i = 0; i < kStatClasses; ++i) {
    ctx->stat_dead[i] = 0;
    ctx->stat_ms[i] = 0.0;
    ctx->stat_flops[i] = 0.0;
    ctx->stat_n[i] = 0;
  }
  return GBI_OK;
}

gbi_status gbi_kernel_stats(gbi_ctx* ctx, int kernel_class, double* total_ms, long long* launches,
                            double* flops) {
  if (!ctx || kernel_class < 0 || kernel_class >= kStatClasses) return GBI_ERR_ARG;
  drain_profile(ctx);
  if (total_ms) *total_ms = ctx->stat_ms[kernel_class];
  const long long live = ctx->stat_n[kernel_class] - (ctx->prof ? ctx->stat_dead[kernel_class] : 0);
  const double per = ctx->stat_n[kernel_class] > 0 ? ctx->stat_flops[kernel_class] / ctx->stat_n[kernel_class] : 0.0;
  if (launches) *launches = live;
  if (flops) *flops = per * double(live);
  return GBI_OK;
}

long long gbi_kernel_launches(gbi_ctx* ctx) { return ctx ? ctx->launches : -1; }

long long gbi_solve_graph_replays(gbi_ctx* ctx) { return ctx ? ctx->solve_replays : -1; }

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
constexpr size_t kOffB = kOffXQ + al256(sizeof(double) * kStaticMaxND);
constexpr size_t kOffR = kOffB + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffDelta = kOffR + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffXVL = kOffDelta + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffKry = kOffXVL + al256(sizeof(double) * 6 * kStaticMaxN);
constexpr size_t kOffW = kOffKry + al256(sizeof(double) * (size_t)(kStaticMaxRestart + 1) * kStaticMaxNH);
constexpr size_t kOffMin = kOffW + al256(sizeof(double) * kStaticMaxNH);
constexpr size_t kOffX32 = kOffMin + 256;
constexpr int kStaticMaxH = 48;           // the largest gbi_h taken here (trunc 4)
// x32: per-sphere source records of a double-float pass over every column, rec_floats(D, df)
// = 2 round4(h + 6) <= 2 (h + 9) floats per sphere, within the limits above
constexpr size_t kStaticX32Floats = 2 * ((size_t)kStaticMaxNH + 9 * (size_t)kStaticMaxN);
constexpr size_t kOffGs = kOffX32 + al256(sizeof(float) * kStaticX32Floats);
// solver state of one system: restart <= 32, at most kStaticMaxH Arnoldi chunks
constexpr size_t kStaticGsDoubles = gstate_doubles(kStaticMaxRestart, 1, kStaticMaxH, kFusedBlocks);
constexpr size_t kOffBoff = kOffGs + al256(sizeof(double) * kStaticGsDoubles);
constexpr size_t kOffBsys = kOffBoff + 256;
constexpr size_t kStaticBytes = kOffBsys + al256(sizeof(int) * kStaticMaxN);
static_assert(arnoldi_chunks(1, kStaticMaxH) == kStaticMaxH, "one system: one chunk per higher component");
static_assert(kStaticBytes < 3u * 1024u * 1024u, "the static scratch stays below 3 MB");
static_assert(((sizeof(GDev) + 15) & ~size_t(15)) + 32 + sizeof(DSolve) + 16 <= 4096,
              "the read-back area holds one system's state, the counters and the device record");

// The scratch itself (about 2.9 MB).  Every device that loads the library holds it
// until the process exits.  Host code must not use this symbol as an address.
__device__ __align__(256) unsigned char g_solve_scratch[kStaticBytes];

constexpr int kStaticMaxDevices = 64;
// device address of the array, per device ordinal, published once looked up
std::atomic<void*> g_scratch_addr[kStaticMaxDevices];
// host copies of the solver state read back by a call (pageable), per device ordinal
alignas(64) char g_static_host[kStaticMaxDevices][4096];

}  // namespace

extern "C" gbi_status gbi_solve_static(void* stream, const gbi_params* prm, int N, const double* R,
                                       const double* Va, const double* Oa, const double* VH, const double* Fe,
                                       const double* Te, double* V, double* Omega, double* QH, int warm_start,
                                       gbi_info* info) {
  if (!valid_params(prm) || N < 0) return GBI_ERR_ARG;
  const int h = gbi_h(prm->trunc);
  if (h > kStaticMaxH || N > kStaticMaxN || (long long)N * h > kStaticMaxNH) return GBI_ERR_ARG;
  if (prm->restart > kStaticMaxRestart) return GBI_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return GBI_ERR_CUDA;
  void* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (addr == nullptr) {
    // set-up on this device: the device address of the static array (two threads that
    // race here look up the same address)
    if (cudaGetSymbolAddress(&addr, g_solve_scratch) != cudaSuccess || addr == nullptr) return GBI_ERR_CUDA;
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  unsigned char* base = static_cast<unsigned char*>(addr);
  gbi_ctx c;
  c.device = dev;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  c.hs = g_static_host[dev];
  c.hs_cap = sizeof(g_static_host[dev]);
  c.allow_graphs = false;      // graph instantiation could allocate
  c.fixed = true;
  auto bind = [&](Buf& b, size_t off, size_t bytes) {
    b.p = base + off;
    b.bytes = bytes;
  };
  bind(c.pos_hi, kOffHi, kOffLo - kOffHi);
  bind(c.pos_lo, kOffLo, kOff64 - kOffLo);
  bind(c.pos64, kOff64, kOffXQ - kOff64);
  bind(c.xQ, kOffXQ, kOffB - kOffXQ);
  bind(c.b, kOffB, kOffR - kOffB);
  bind(c.r, kOffR, kOffDelta - kOffR);
  bind(c.delta, kOffDelta, kOffXVL - kOffDelta);
  bind(c.xVL, kOffXVL, kOffKry - kOffXVL);
  bind(c.krylov, kOffKry, kOffW - kOffKry);
  bind(c.w, kOffW, kOffMin - kOffW);
  bind(c.minr2, kOffMin, 256);
  bind(c.x32, kOffX32, kOffGs - kOffX32);
  bind(c.gstate, kOffGs, kOffBoff - kOffGs);
  bind(c.boff, kOffBoff, 256);
  bind(c.bsys, kOffBsys, kStaticBytes - kOffBsys);
  gbi_params p = *prm;
  if (p.restart <= 0) p.restart = kStaticMaxRestart;
  return gbi_solve(&c, &p, N, R, Va, Oa, VH, Fe, Te, V, Omega, QH, warm_start, info);
}
