// C ABI of the learned near-field correction: neighbour lists, network weights,
// inference, labels and training (kernels in mlp_kernel.cu and mlp_tc.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"

namespace gbi {
namespace {

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


// Network inference with the selected engine.  The tcgen05 kernel reports a wait that
// gave up through a device flag that gbi_mlp_status reads back.
gbi_status mlp_infer(gbi_ctx* ctx, int np_, const float* F, const float* FR, float* out) {
  if (ctx->mlp_engine == 1) {
    GBI_CHECK(mlpk::infer_tc(np_, F, FR, ctx->mlp_pk_tc.p, out, P<int>(ctx->mlp_err), sm_count(ctx), ctx->mlp_head,
                             ctx->stream));
    ++ctx->launches;
    return GBI_OK;
  }
  GBI_CHECK(mlpk::infer(np_, F, FR, ctx->mlp_pk.p, out, sm_count(ctx), ctx->mlp_head, ctx->stream));
  ++ctx->launches;
  return GBI_OK;
}

}  // namespace
}  // namespace gbi

using namespace gbi;

extern "C" {

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

gbi_status gbi_mlp_set_head(gbi_ctx* ctx, int head) {
  if (!ctx || (head != mlpk::HEAD_VELOCITY && head != mlpk::HEAD_QSTRAIN)) return GBI_ERR_ARG;
  ctx->mlp_head = head;
  return GBI_OK;
}

gbi_status gbi_mlp_correct(gbi_ctx* ctx, int N, const double* R, const double* p, double a, double s0, int nsys,
                           const int* offsets_host, double* V, double* Omega, int* npairs) {
  if (!ctx || N < 0 || !(a > 0) || nsys < 0 || (nsys > 1 && !offsets_host)) return GBI_ERR_ARG;
  if (nsys > 1 && (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N)) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  if (ctx->mlp_head != mlpk::HEAD_VELOCITY) {
    ctx->err = "gbi_mlp_correct needs the velocity head (gbi_mlp_set_head 0)";
    return GBI_ERR_ARG;
  }
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

gbi_status gbi_mlp_correct_qh(gbi_ctx* ctx, int N, const double* R, const double* p, double a, double s0, int nsys,
                              const int* offsets_host, int h, double* QH, int* npairs) {
  if (!ctx || N < 0 || !(a > 0) || nsys < 0 || (nsys > 1 && !offsets_host) || h < 5) return GBI_ERR_ARG;
  if (nsys > 1 && (!valid_offsets(nsys, offsets_host) || offsets_host[nsys] != N)) return GBI_ERR_ARG;
  GBI_TRY(mlp_require(ctx));
  if (ctx->mlp_head != mlpk::HEAD_QSTRAIN) {
    ctx->err = "gbi_mlp_correct_qh needs the strain-mode head (gbi_mlp_set_head 1)";
    return GBI_ERR_ARG;
  }
  if (npairs) *npairs = 0;
  if (N == 0) return GBI_OK;
  if (!R || !p || !QH) return GBI_ERR_ARG;
  int np_ = 0;
  GBI_TRY(mlp_prepare(ctx, N, R, p, a, nsys, offsets_host, np_));
  GBI_TRY(mlp_infer(ctx, np_, P<float>(ctx->mf_F), P<float>(ctx->mf_FR), P<float>(ctx->mf_lab)));
  GBI_CHECK(mlpk::sphere_sums_q(N, P<int>(ctx->nb_start), P<float>(ctx->mf_lab), s0 / ctx->mlp_sigma, QH, h,
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
                              ctx->mlp_head, ctx->mlp_engine, ctx->mlp_pk_tc.p, P<int>(ctx->mlp_err), sm_count(ctx),
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

gbi_status gbi_mlp_labels_qh(gbi_ctx* ctx, int N, int h, double s0, const double* QHx, const double* QH1,
                             double* sigma, double* labels) {
  if (!ctx || N <= 0 || h < 5 || !(s0 != 0) || !QHx || !QH1 || !sigma || !labels) return GBI_ERR_ARG;
  if (!(*sigma > 0)) {
    // sigma = the power of two nearest to 1 / rms of (exact - one-body) / s0 over 6 N numbers
    const int nb = (N + 255) / 256;
    GBI_TRY(ensure(ctx, ctx->mf_loss, sizeof(double) * (size_t)(nb + 1)));
    GBI_CHECK(mlpk::labels_q(N, h, s0, 1.0, QHx, QH1, nullptr, P<double>(ctx->mf_loss), ctx->stream));
    GBI_CHECK(mlpk::sum_into(P<double>(ctx->mf_loss), nb, P<double>(ctx->mf_loss) + nb, ctx->stream));
    ctx->launches += 2;
    double sq = 0.0;
    GBI_CHECK(cudaMemcpyAsync(&sq, P<double>(ctx->mf_loss) + nb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
    const double rms = std::sqrt(sq / (6.0 * N));
    if (!(rms > 0)) return GBI_ERR_ARG;
    *sigma = std::ldexp(1.0, (int)std::lround(-std::log2(rms)));
  }
  GBI_CHECK(mlpk::labels_q(N, h, s0, *sigma, QHx, QH1, labels, nullptr, ctx->stream));
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
                                  P<float>(ctx->mlp_grad), ctx->mlp_head, ctx->mlp_engine, ctx->mlp_pk_tc.p,
                                  P<int>(ctx->mlp_err), sm_count(ctx), ctx->stream));
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

}  // extern "C"
