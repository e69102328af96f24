// Flow field of the Galerkin representation at points in the fluid (Sec. III,
// Eq. flow_expression and Eq. galerkin_representation_flow_yl): after a solve, the
// exterior flow at any point x is
//
//   v(x) = -(1 / (8 pi eta)) sum_m [F^l' grad^(l') G](x - R_m) . Q_m,   Q^L = F^L,
//
// the single-layer flow of every sphere's modes with its flow coefficients Q (the
// exterior double-layer flow of each mode is a single-layer flow of the same mode).
// Each (point, sphere) term is the 1s row of the pair operator for a target of radius
// zero (pair_body with the SET_P rows): the finite-size operator of the target drops out
// and the source keeps its own, 1 + a^2/(4l'+6) lap.
//
// Kernel: one thread per point, 128 points per block; all threads of a block walk the
// same spheres, staged in shared memory in tiles of 64 (broadcast reads).  FP32 (records
// of every column, two-float centres) or FP64.  Points inside a sphere (|x - R_m| < a)
// get NaN: the representation holds in the fluid only.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>

#include "ctx.cuh"
#include "pair_kernel.cuh"

namespace gbi {
namespace {

constexpr int kFlowThreads = 128;
constexpr int kFlowTile = 64;

struct FlowArgs {
  int N, M;
  double a;
  double scale;          // -1 / (8 pi eta a)
  Positions pos;         // sphere centres
  const float* rec;      // FP32: per-sphere records of every column (rec_floats(D, false) floats)
  const double* x;       // FP64: coefficients, component-major [D][N]
  const double* X;       // points [M][3]
  double* U;             // flow [M][3]
  int* inside;           // points found inside a sphere (count)
};

template <int TR, typename T>
__global__ void __launch_bounds__(kFlowThreads) k_flow(const FlowArgs f) {
  using S = PassShape<TR, SET_P, SET_ALL>;
  constexpr int D = S::D;
  constexpr bool F32 = std::is_same<T, float>::value;
  constexpr int NCP = RecShape<D>::NCP;
  constexpr int RECF = F32 ? NCP : D;            // floats (FP32) or doubles per staged sphere
  __shared__ __align__(16) T s_x[kFlowTile * RECF];
  __shared__ __align__(16) T s_p[kFlowTile * 8];  // hi xyz, lo xyz (FP32) or xyz (FP64)

  const int i = blockIdx.x * kFlowThreads + threadIdx.x;
  const bool live = i < f.M;
  double X[3] = {0.0, 0.0, 0.0};
  if (live) {
    X[0] = f.X[3 * (size_t)i];
    X[1] = f.X[3 * (size_t)i + 1];
    X[2] = f.X[3 * (size_t)i + 2];
  }
  T ph[3], pl[3];
  for (int c = 0; c < 3; ++c) {
    if constexpr (F32) {
      ph[c] = float(X[c]);
      pl[c] = float(X[c] - double(ph[c]));
    } else {
      ph[c] = X[c];
      pl[c] = 0.0;
    }
  }
  const T a = T(f.a);
  const T a2 = a * a;
  T acc[3] = {T(0), T(0), T(0)};
  bool inside = false;
  for (int base = 0; base < f.N; base += kFlowTile) {
    const int len = min(kFlowTile, f.N - base);
    __syncthreads();
    for (int k = threadIdx.x; k < len * RECF; k += kFlowThreads) {
      const int j = k / RECF, q = k - j * RECF;
      if constexpr (F32) s_x[k] = f.rec[(size_t)(base + j) * NCP + q];
      else s_x[k] = f.x[(size_t)q * f.N + base + j];
    }
    for (int j = threadIdx.x; j < len; j += kFlowThreads) {
      if constexpr (F32) {
        const float4 h = f.pos.hi[base + j], l = f.pos.lo[base + j];
        s_p[8 * j] = h.x; s_p[8 * j + 1] = h.y; s_p[8 * j + 2] = h.z;
        s_p[8 * j + 3] = l.x; s_p[8 * j + 4] = l.y; s_p[8 * j + 5] = l.z;
      } else {
        const dpos4 p = f.pos.p64[base + j];
        s_p[8 * j] = p.x; s_p[8 * j + 1] = p.y; s_p[8 * j + 2] = p.z;
        s_p[8 * j + 3] = 0.0; s_p[8 * j + 4] = 0.0; s_p[8 * j + 5] = 0.0;
      }
    }
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < len; ++j) {
      const T* sp = s_p + 8 * j;
      const T dx = (ph[0] - sp[0]) + (pl[0] - sp[3]);
      const T dy = (ph[1] - sp[1]) + (pl[1] - sp[4]);
      const T dz = (ph[2] - sp[2]) + (pl[2] - sp[5]);
      if (dx * dx + dy * dy + dz * dz < a2) {
        inside = true;
        continue;
      }
      T xl[D];
#pragma unroll
      for (int q = 0; q < D; ++q) xl[q] = s_x[j * RECF + q];
      pair_body<TR, SET_P, SET_ALL, T>(dx, dy, dz, a, xl, acc);
    }
  }
  if (!live) return;
  double* u = f.U + 3 * (size_t)i;
  if (inside) {
    u[0] = u[1] = u[2] = __longlong_as_double(0x7ff8000000000000ll);
    atomicAdd(f.inside, 1);
    return;
  }
  // 1s components are ordered (y, z, x)
  u[0] = f.scale * double(acc[2]);
  u[1] = f.scale * double(acc[0]);
  u[2] = f.scale * double(acc[1]);
}

template <int TR>
cudaError_t launch_flow_t(bool fp32, const FlowArgs& f, cudaStream_t st) {
  const dim3 grid((f.M + kFlowThreads - 1) / kFlowThreads);
  if constexpr (TR == 5 || TR == 40) {
    // l <= 5 and the minimal set: FP64 only
    if (fp32) return cudaErrorInvalidValue;
    k_flow<TR, double><<<grid, kFlowThreads, 0, st>>>(f);
  } else {
    if (fp32) k_flow<TR, float><<<grid, kFlowThreads, 0, st>>>(f);
    else k_flow<TR, double><<<grid, kFlowThreads, 0, st>>>(f);
  }
  return cudaGetLastError();
}

double flops_point(int trunc) {
  switch (trunc) {
    case 2: return gbi_t2_flops_point;
    case 3: return gbi_t3_flops_point;
    case 4: return gbi_t4_flops_point;
    case 5: return gbi_t5_flops_point;
    default: return gbi_t40_flops_point;
  }
}

}  // namespace
}  // namespace gbi

using namespace gbi;

extern "C" gbi_status gbi_flow(gbi_ctx* ctx, const gbi_params* prm, int N, const double* R, const double* Fe,
                               const double* Te, const double* QH, int M, const double* X, double* U,
                               int* n_inside) {
  if (!ctx || !valid_params(prm) || N < 0 || M < 0) return GBI_ERR_ARG;
  if (n_inside) *n_inside = 0;
  if (M == 0) return GBI_OK;
  if (!X || !U || (N > 0 && (!R || !Fe || !Te || !QH))) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  Setup s;
  GBI_TRY(setup_call(ctx, s, N, prm->trunc, prm->a, prm->eta, R));
  const int D = s.D, h = s.h;
  const bool fp32 = prm->precision != 0;
  GBI_TRY(ensure(ctx, ctx->flowx, sizeof(double) * (size_t)D * (N > 0 ? N : 1)));
  GBI_TRY(ensure(ctx, ctx->flowcnt, sizeof(int)));
  GBI_CHECK(cudaMemsetAsync(ctx->flowcnt.p, 0, sizeof(int), ctx->stream));
  double* x = P<double>(ctx->flowx);
  FlowArgs f;
  f.N = N;
  f.M = M;
  f.a = s.a;
  f.scale = -1.0 / (8.0 * kPi * s.eta * s.a);
  f.pos = s.pos;
  f.rec = nullptr;
  f.x = x;
  f.X = X;
  f.U = U;
  f.inside = P<int>(ctx->flowcnt);
  if (N > 0) {
    // F^L and Q^H in internal coordinates, component-major [D][N]
    Scales hscale;
    for (int i = 0; i < kMaxD; ++i) hscale.v[i] = (i < h) ? s.scale.v[6 + i] : 1.0;
    k_pack_lower<<<grid1(N), 256, 0, ctx->stream>>>(N, s.a, s.scale.v[3], Fe, Te, x, nullptr);
    k_pack_higher<<<grid1((size_t)N * h), 256, 0, ctx->stream>>>(N, h, QH, hscale, 1.0, x + (size_t)6 * N, nullptr);
    ctx->launches += 2;
    GBI_CHECK(cudaGetLastError());
    if (fp32) {
      GBI_TRY(ensure(ctx, ctx->flowrec, sizeof(float) * rec_floats(D, false) * (size_t)N));
      ColScale cs;
      for (int i = 0; i < kMaxD; ++i) cs.v[i] = 1.0;
      GBI_CHECK(launch_records(false, N, D, x, nullptr, 0, nullptr, cs, P<float>(ctx->flowrec), ctx->stream));
      ++ctx->launches;
      f.rec = P<float>(ctx->flowrec);
    }
  }
  const double flops = flops_point(prm->trunc) * double(N) * double(M);
  cudaError_t e = timed(ctx, fp32 ? 30 : 29, flops, 1, [&] {
    switch (prm->trunc) {
      case 2: return launch_flow_t<2>(fp32, f, ctx->stream);
      case 3: return launch_flow_t<3>(fp32, f, ctx->stream);
      case 4: return launch_flow_t<4>(fp32, f, ctx->stream);
      case 5: return launch_flow_t<5>(fp32, f, ctx->stream);
      default: return launch_flow_t<40>(fp32, f, ctx->stream);
    }
  });
  GBI_CHECK(e);
  if (n_inside) {
    GBI_CHECK(cudaMemcpyAsync(n_inside, ctx->flowcnt.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  }
  return GBI_OK;
}
