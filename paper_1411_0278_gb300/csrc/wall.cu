// Spheres above a plane no-slip wall (z = 0, fluid z > 0): the superposition
// approximation of Sec. IV with the wall's Green's function in place of the Oseen tensor
// (Sec. VI: another geometry enters through its Green's function).
//
// Blake's Green's function is the Oseen tensor plus an image system at
// y* = (y1, y2, -y3), h = y3, R = x - y*, m = (1, 1, -1):
//
//   W_ij(x, y) = -G_ij(R) + 2 h m_j [ h (d_ij/|R|^3 - 3 R_i R_j/|R|^5) + d_i3 R_j/|R|^3
//                                      - (d_ij R_3 + R_i d_j3)/|R|^3 + 3 R_i R_3 R_j/|R|^5 ].
//
// gbi_wall_superpose adds to the unbounded superposition (gbi_superpose, l <= 2) the image
// flows, at the point-singularity level, of every sphere's force F, torque T and
// stresslet S = (20/3) pi eta a^2 V^(2s) (what it exerts on the fluid), its own images
// included:
//
//   8 pi eta u(x) = sum_m W_ij(x, R_m) F_j + D_jk d/dy_k W_ij(x, y)|_{y = R_m},
//   D_jk = S_jk + (1/2) eps_kjl T_l,   V_n += u(R_n),   Omega_n += curl u (R_n) / 2.
//
// Derivatives are exact (to rounding): forward-mode dual numbers, nested.  The inner
// level carries the three directional derivatives along the rows D_j. of the source's
// dipole tensor (so its j-th component is D_jk d/dy_k), the outer one the derivatives
// along the three axes at the target (for the curl).  One thread per target; sources in
// shared-memory tiles; the sources are split over gridDim.y slices whose partial sums are
// added in slice order by a second kernel, so the result does not depend on timing.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "ctx.cuh"
#include "gbi_generated.cuh"

namespace gbi {
namespace {

constexpr int kWallThreads = 128;
constexpr int kWallTile = 64;
constexpr int kWallRec = 16;   // per source: x y z, F (3), D (9, row-major), pad

// Flops of one (target, source) term (FMA = 2) as the compiled FP32 kernel executes them:
// 392.6 FFMA and 696 other FP32 instructions per term (ncu instruction statistics of the
// N = 10^4 launch).  The nested dual numbers as written would count 4 096 -- a D2 product
// is 82 flops -- but most derivative entries are structurally zero (the target-side
// derivatives of the source height, the constant derivatives of R) and fold away.
constexpr int kWallPairFlops = 1481;

// ---------------------------------------------------------------------------------
// dual numbers: a value and its derivatives along three directions.  D1 = Dual3<T>
// (inner, source side), D2 = Dual3<D1> (outer, target side).
// ---------------------------------------------------------------------------------
template <typename U> struct Dual3 {
  U v;
  U d[3];
};

template <typename U> __device__ __forceinline__ Dual3<U> operator+(const Dual3<U>& a, const Dual3<U>& b) {
  Dual3<U> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <typename U> __device__ __forceinline__ Dual3<U> operator-(const Dual3<U>& a, const Dual3<U>& b) {
  Dual3<U> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <typename U> __device__ __forceinline__ Dual3<U> operator*(const Dual3<U>& a, const Dual3<U>& b) {
  Dual3<U> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = a.v * b.d[k] + a.d[k] * b.v;
  return r;
}
// scaling by a plain number
template <typename U, typename T, typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
__device__ __forceinline__ Dual3<U> operator*(T s, const Dual3<U>& a) {
  Dual3<U> r;
  r.v = s * a.v;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = s * a.d[k];
  return r;
}

__device__ __forceinline__ float wall_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double wall_rsqrt(double x) { return rsqrt(x); }

// a^(-1/2) and its derivatives: (a^-1/2)' = -1/2 a^-3/2
template <typename T> __device__ __forceinline__ Dual3<T> rsqrt1(const Dual3<T>& a) {
  Dual3<T> r;
  r.v = wall_rsqrt(a.v);
  const T f1 = T(-0.5) * r.v * r.v * r.v;
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = f1 * a.d[k];
  return r;
}
template <typename T> __device__ __forceinline__ Dual3<Dual3<T>> rsqrt2(const Dual3<Dual3<T>>& a) {
  Dual3<Dual3<T>> r;
  r.v = rsqrt1(a.v);
  const Dual3<T> f1 = T(-0.5) * (r.v * r.v * r.v);
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[k] = f1 * a.d[k];
  return r;
}

template <typename T> __device__ __forceinline__ Dual3<T> d1_const(T v) {
  Dual3<T> r;
  r.v = v;
  r.d[0] = r.d[1] = r.d[2] = T(0);
  return r;
}
template <typename T> __device__ __forceinline__ Dual3<Dual3<T>> d2_const(T v) {
  Dual3<Dual3<T>> r;
  r.v = d1_const(v);
  r.d[0] = r.d[1] = r.d[2] = d1_const(T(0));
  return r;
}

// Image flow at target x (times 8 pi eta) of a source at y with force F and dipole D:
// u_i += W_ij F_j + D_jk dW_ij/dy_k, and the derivatives du_i/dx_l into the curl c.
template <typename T>
__device__ __forceinline__ void wall_image_pair(const T* x, const T* src, T* u, T* c) {
  using D1 = Dual3<T>;
  using D2 = Dual3<D1>;
  const T* y = src;
  const T* F = src + 3;
  const T* D = src + 6;   // D[3 j + k] = D_jk
  // R_k = x_k - y*_k: outer derivative d/dx_l = delta_kl, inner (direction j) derivative
  // D_jk dR_k/dy_k = -D_jk (k = 0, 1) or +D_j2 (k = 2: R_3 = x_3 + y_3)
  D2 R[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T sgn = k == 2 ? T(1) : T(-1);
    R[k].v.v = k == 2 ? x[2] + y[2] : x[k] - y[k];
#pragma unroll
    for (int j = 0; j < 3; ++j) R[k].v.d[j] = sgn * D[3 * j + k];
#pragma unroll
    for (int l = 0; l < 3; ++l) R[k].d[l] = d1_const(l == k ? T(1) : T(0));
  }
  // h = y_3: inner derivative D_j2, no outer derivative
  D2 h = d2_const(y[2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) h.v.d[j] = D[3 * j + 2];
  // shared factors (D2 products: 6 + 3 + 1 + 1 + 3 = 14; sums and scalings: 2 + 1 + 1)
  D2 RR[6];                                         // R_i R_j, i <= j
  RR[0] = R[0] * R[0];
  RR[1] = R[0] * R[1];
  RR[2] = R[0] * R[2];
  RR[3] = R[1] * R[1];
  RR[4] = R[1] * R[2];
  RR[5] = R[2] * R[2];
  const D2 iR = rsqrt2(RR[0] + RR[3] + RR[5]);
  const D2 iR2 = iR * iR;
  const D2 iR3 = iR2 * iR;
  const D2 iR5 = iR3 * iR2;
  const D2 hR3 = h * iR3;
  const D2 c5 = T(3) * ((R[2] - h) * iR5);          // 3 (R_3 - h) / |R|^5
  D2 RiR3[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) RiR3[k] = R[k] * iR3;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int lo = i < j ? i : j, hi = i < j ? j : i;
      const D2& Rij = RR[lo == 0 ? hi : (lo == 1 ? 2 + hi : 5)];
      // Oseen tensor at R, and the bracket of the image terms (per entry: 3 D2 products,
      // up to 4 sums and 1 scaling)
      D2 g = Rij * iR3;
      D2 t = Rij * c5;
      if (i == j) {
        g = g + iR;
        t = t + hR3 - RiR3[2];
      }
      if (i == 2) t = t + RiR3[j];
      if (j == 2) t = t - RiR3[i];
      const D2 w = T(2 * (j == 2 ? -1 : 1)) * (h * t) - g;
      u[i] += w.v.v * F[j] + w.v.d[j];
      // du_i/dx_l = w.d[l].v F_j + w.d[l].d[j]; curl c = (d2u3 - d3u2, d3u1 - d1u3, d1u2 - d2u1)
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        const T dl = w.d[l].v * F[j] + w.d[l].d[j];
        if (i == 2 && l == 1) c[0] += dl;
        if (i == 1 && l == 2) c[0] -= dl;
        if (i == 0 && l == 2) c[1] += dl;
        if (i == 2 && l == 0) c[1] -= dl;
        if (i == 1 && l == 0) c[2] += dl;
        if (i == 0 && l == 1) c[2] -= dl;
      }
    }
  }
}

// Source records: position, force, dipole D = S + A(T) in T.
template <typename T>
__global__ void k_wall_records(int N, double a, double eta, const double* __restrict__ R,
                               const double* __restrict__ VH, int h, const double* __restrict__ Fe,
                               const double* __restrict__ Te, T* __restrict__ rec) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  T* o = rec + (size_t)m * kWallRec;
  const double cs = (20.0 / 3.0) * kPi * eta * a * a;
  double s6[6];   // xx xy xz yy yz zz of the packed V^(2s)
  gbi_unpack2<double>(VH + (size_t)h * m, s6);
  const double S[9] = {s6[0], s6[1], s6[2], s6[1], s6[3], s6[4], s6[2], s6[4], s6[5]};
  const double T0 = Te[3 * (size_t)m], T1 = Te[3 * (size_t)m + 1], T2 = Te[3 * (size_t)m + 2];
  // A_jk = (1/2) eps_kjl T_l
  const double A[9] = {0.0, -0.5 * T2, 0.5 * T1, 0.5 * T2, 0.0, -0.5 * T0, -0.5 * T1, 0.5 * T0, 0.0};
  for (int k = 0; k < 3; ++k) {
    o[k] = T(R[3 * (size_t)m + k]);
    o[3 + k] = T(Fe[3 * (size_t)m + k]);
  }
  for (int q = 0; q < 9; ++q) o[6 + q] = T(cs * S[q] + A[q]);
  o[15] = T(0);
}

// Partial image sums of the targets over the sources of slice blockIdx.y.
template <typename T>
__global__ void __launch_bounds__(kWallThreads) k_wall_pairs(int N, int per_slice, const T* __restrict__ rec,
                                                             T* __restrict__ part) {
  __shared__ T s_rec[kWallTile * kWallRec];
  const int n = blockIdx.x * kWallThreads + threadIdx.x;
  const int m0 = blockIdx.y * per_slice;
  const int m1 = min(N, m0 + per_slice);
  T x[3] = {T(0), T(0), T(0)};
  if (n < N)
    for (int k = 0; k < 3; ++k) x[k] = rec[(size_t)n * kWallRec + k];
  T u[3] = {T(0), T(0), T(0)}, c[3] = {T(0), T(0), T(0)};
  for (int base = m0; base < m1; base += kWallTile) {
    const int len = min(kWallTile, m1 - base);
    __syncthreads();
    for (int q = threadIdx.x; q < len * kWallRec; q += kWallThreads) s_rec[q] = rec[(size_t)base * kWallRec + q];
    __syncthreads();
    if (n < N)
      for (int j = 0; j < len; ++j) wall_image_pair<T>(x, s_rec + j * kWallRec, u, c);
  }
  if (n < N) {
    T* o = part + ((size_t)blockIdx.y * N + n) * 6;
    for (int k = 0; k < 3; ++k) {
      o[k] = u[k];
      o[3 + k] = c[k];
    }
  }
}

// V += u / (8 pi eta), Omega += c / (16 pi eta), the slices added in order.
template <typename T>
__global__ void k_wall_reduce(int N, int slices, double eta, const T* __restrict__ part, double* V, double* Om) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int q = 0; q < slices; ++q)
    for (int k = 0; k < 6; ++k) s[k] += double(part[((size_t)q * N + n) * 6 + k]);
  const double f = 1.0 / (8.0 * kPi * eta);
  for (int k = 0; k < 3; ++k) {
    V[3 * (size_t)n + k] += f * s[k];
    Om[3 * (size_t)n + k] += 0.5 * f * s[3 + k];
  }
}

int wall_slices(int N) {
  // about four blocks per SM on 152 SMs, at least 32 sources per slice
  const int tb = (N + kWallThreads - 1) / kWallThreads;
  int s = (608 + tb - 1) / tb;
  const int maxs = (N + 31) / 32;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

template <typename T>
cudaError_t launch_wall_t(int N, double a, double eta, const double* R, const double* VH, int h, const double* Fe,
                          const double* Te, double* V, double* Om, void* scratch, cudaStream_t st) {
  T* rec = static_cast<T*>(scratch);
  const int slices = wall_slices(N);
  const int per = (N + slices - 1) / slices;
  T* part = rec + (size_t)N * kWallRec;
  k_wall_records<T><<<(N + 255) / 256, 256, 0, st>>>(N, a, eta, R, VH, h, Fe, Te, rec);
  k_wall_pairs<T><<<dim3((N + kWallThreads - 1) / kWallThreads, slices), kWallThreads, 0, st>>>(N, per, rec, part);
  k_wall_reduce<T><<<(N + 255) / 256, 256, 0, st>>>(N, slices, eta, part, V, Om);
  return cudaGetLastError();
}

size_t wall_scratch_bytes(int N, bool fp32) {
  const size_t w = fp32 ? sizeof(float) : sizeof(double);
  return w * ((size_t)N * kWallRec + (size_t)wall_slices(N) * N * 6) + 256;
}

}  // namespace
}  // namespace gbi

using namespace gbi;

extern "C" gbi_status gbi_wall_superpose(gbi_ctx* ctx, const gbi_params* prm, int N, const double* R,
                                         const double* Va, const double* Oa, const double* VH, const double* Fe,
                                         const double* Te, double* V, double* Omega) {
  if (!ctx || !valid_params(prm) || N < 0 || prm->trunc != 2) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Oa || !VH || !Fe || !Te || !V || !Omega) return GBI_ERR_ARG;
  // the unbounded superposition first (direct pairs with their finite-size terms)
  GBI_TRY(gbi_superpose(ctx, prm, N, R, Va, Oa, VH, Fe, Te, V, Omega));
  cudaSetDevice(ctx->device);
  const bool fp32 = prm->precision != 0 && prm->precision != 2;
  GBI_TRY(ensure(ctx, ctx->wallbuf, wall_scratch_bytes(N, fp32)));
  const int h = gbi_h(prm->trunc);
  const double flops = double(kWallPairFlops) * double(N) * double(N);
  const cudaError_t e = timed(ctx, fp32 ? 32 : 31, flops, 3, [&] {
    return fp32 ? launch_wall_t<float>(N, prm->a, prm->eta, R, VH, h, Fe, Te, V, Omega, ctx->wallbuf.p, ctx->stream)
                : launch_wall_t<double>(N, prm->a, prm->eta, R, VH, h, Fe, Te, V, Omega, ctx->wallbuf.p,
                                        ctx->stream);
  });
  GBI_CHECK(e);
  return GBI_OK;
}
