// Spheres in a periodic cube of side L: the point-force superposition with the periodic
// Green's function, summed by Ewald's method (Sec. VI: in a periodic domain the flow sum
// converges only conditionally and needs a limiting procedure; this is Hasimoto's, zero
// mean flow over the cell, the k = 0 term left out).
//
// With G = (d_ij lap - d_i d_j) r (u = G F / (8 pi eta)) and the split r = r erfc(xi r) +
// r erf(xi r):
//   real space   G^real F = (f'' + f'/r) F - (f'' - f'/r) (r.F) r / r^2,  f = r erfc(xi r),
//                f' = erfc(xi r) - (2 xi r / sqrt pi) e^{-xi^2 r^2},
//                f'' = (4 xi / sqrt pi) (xi^2 r^2 - 1) e^{-xi^2 r^2};
//   wave space   G^rec(k) = 8 pi (d - k k / k^2) / k^2 (1 + q + 2 q^2) e^{-q},  q = k^2/(4 xi^2);
//   8 pi eta u_n = sum_{m != n, |r| < rc} G^real(r_nm) F_m
//                + (2 / L^3) sum_{k in a half space} Re[ G^rec(k) S(k) e^{i k.R_n} ]
//                - (8 xi / sqrt pi) F_n,     S(k) = sum_m F_m e^{-i k.R_m},
// and V_n = V^a_n + F_n / (6 pi eta a) + u_n.  The last term of u_n removes the singular
// direct term of the sphere's own contribution (the limit of G - G^real at r = 0), so its
// own periodic images remain.
//
// The split parameter balances the two sums: the cube is cut into M^3 cells of side
// rc = L / M (M >= 3; M = 0 means every pair by the minimum image, rc = L / 2) and
// xi = c_r / rc, the wave vectors kept up to |k| = 2 xi sqrt(q_max), with (c_r, q_max) =
// (4.2, 30) in FP32 and (5.6, 40) in FP64.  The real-space, wave-space and self parts
// cancel to a small net velocity, so the truncation must sit well below the target:
// these give ~1e-6 (FP32, whose accumulations are also compensated) and ~1e-13 of the
// velocities.  M minimises the estimated work 27 N^2 / M^3 (pairs) + 2 N n_k (wave terms),
// so the cost grows as N^1.5 instead of N^2.  Real space: a cell list (cells sorted by a
// stable radix sort, so every sum runs in a fixed order), one thread per target over the
// 27 neighbouring cells; wave space: the structure factors S(k), one thread per k over
// all spheres, then one thread per target over all k.  No step depends on timing.
//
// Positions enter as fractions s = x / L of the cell.  In FP32 a separation is formed as
// (hi_n - hi_m) + (lo_n - lo_m) of a two-float split of s, wrapped to the nearest image
// (exact in the cell's units) and only then scaled by L; a phase k.R = 2 pi m.s is taken
// as frac(m.s15) + m.s_rem, s15 = s rounded to 15 bits (so m.s15 is exact for |m_i| <=
// 127) and s_rem the rest, then sin / cos of 2 pi times that -- no large argument is
// rounded.  FP64 uses s itself.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ctx.cuh"

namespace gbi {
namespace {

constexpr int kPerThreads = 128;
constexpr int kPerTile = 128;
constexpr double kSqrtPi = 1.7724538509055160273;

struct EwaldPlan {
  int M = 0;          // cells per side (0: all pairs, minimum image)
  double rc = 0, xi = 0, kc = 0;
  int mmax = 0;       // |m_i| <= mmax for k = 2 pi m / L
  long long nk = 0;   // wave vectors kept (half space)
};

// the FP32 phases need |m_i| <= 127 (mmax is about 7.3 M there)
inline int ewald_max_cells(bool fp32) { return fp32 ? 17 : 128; }

EwaldPlan ewald_plan_for(int M, double L, bool fp32) {
  const double cr = fp32 ? 4.2 : 5.6, qmax = fp32 ? 30.0 : 40.0;
  EwaldPlan p;
  p.M = M;
  p.rc = M == 0 ? 0.5 * L : L / M;
  p.xi = cr / p.rc;
  p.kc = 2.0 * p.xi * std::sqrt(qmax);
  p.mmax = (int)std::floor(p.kc * L / (2.0 * kPi));
  const double r = p.kc * L / (2.0 * kPi);
  p.nk = (long long)((2.0 * kPi / 3.0) * r * r * r);   // estimate (the list counts exactly)
  return p;
}

// force_cells: > 0 a given number of cells per side (at least 3), < 0 every pair, 0 the
// cheapest by the work estimate
EwaldPlan ewald_plan(int N, double L, bool fp32, int force_cells) {
  if (force_cells < 0) return ewald_plan_for(0, L, fp32);
  if (force_cells > 0) return ewald_plan_for(std::max(3, std::min(force_cells, ewald_max_cells(fp32))), L, fp32);
  EwaldPlan best = ewald_plan_for(0, L, fp32);
  double best_cost = double(N) * N + 2.0 * N * double(best.nk);
  for (int M = 3; M <= ewald_max_cells(fp32); ++M) {
    const EwaldPlan p = ewald_plan_for(M, L, fp32);
    if (p.nk > 4000000 || (long long)M * M * M > 4 * (long long)std::max(N, 1)) break;
    const double cost = 27.0 * double(N) * N / (double(M) * M * M) + 2.0 * N * double(p.nk);
    if (cost < best_cost) {
      best = p;
      best_cost = cost;
    }
  }
  return best;
}

// the kept wave vectors (half space, |k| <= kc): the integers m (k = 2 pi m / L) and the
// prefactor (2 / L^3) of G^rec
template <typename T> void ewald_kvectors(const EwaldPlan& p, double L, std::vector<T>& out) {
  out.clear();
  const int mm = p.mmax;
  const double s = 2.0 * kPi / L;
  for (int mx = 0; mx <= mm; ++mx)
    for (int my = -mm; my <= mm; ++my)
      for (int mz = -mm; mz <= mm; ++mz) {
        if (mx == 0 && (my < 0 || (my == 0 && mz <= 0))) continue;   // one of each pair +-k
        const double kx = s * mx, ky = s * my, kz = s * mz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        if (k2 > p.kc * p.kc) continue;
        const double q = k2 / (4.0 * p.xi * p.xi);
        const double pref = 2.0 / (L * L * L) * 8.0 * kPi / k2 * (1.0 + q + 2.0 * q * q) * std::exp(-q);
        out.push_back(T(mx));
        out.push_back(T(my));
        out.push_back(T(mz));
        out.push_back(T(pref));
      }
}

__device__ __forceinline__ float per_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double per_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float per_exp(float x) { return expf(x); }
__device__ __forceinline__ double per_exp(double x) { return exp(x); }
// sin and cos of 2 pi f
__device__ __forceinline__ void per_sincos2pi(float f, float* s, float* c) { sincospif(2.0f * f, s, c); }
__device__ __forceinline__ void per_sincos2pi(double f, double* s, double* c) { sincospi(2.0 * f, s, c); }
__device__ __forceinline__ float per_floor(float x) { return floorf(x); }
__device__ __forceinline__ double per_floor(double x) { return floor(x); }
__device__ __forceinline__ float per_rint(float x) { return rintf(x); }
__device__ __forceinline__ double per_rint(double x) { return rint(x); }

// Per sphere: pos[16] = s_hi (3), 0, s_lo (3), 0, s15 (3), 0, s_rem (3), 0 of the cell
// fraction s in [0, 1) (FP64: s, 0, s, 0); frc[4] = F, 0; the cell key.
template <typename T>
__global__ void k_per_records(int N, double L, int M, const double* __restrict__ R, const double* __restrict__ F,
                              T* __restrict__ pos, T* __restrict__ frc, unsigned int* __restrict__ key,
                              int* __restrict__ idx) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  constexpr bool F32 = std::is_same<T, float>::value;
  T* o = pos + 16 * (size_t)n;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double sd = R[3 * (size_t)n + d] / L;
    sd -= floor(sd);                        // into [0, 1)
    if (!(sd < 1.0)) sd = 0.0;              // rounding up to 1
    if (F32) {
      const float hi = float(sd);
      const float s15 = float(floor(sd * 32768.0) / 32768.0);
      o[d] = T(hi);
      o[4 + d] = T(float(sd - double(hi)));
      o[8 + d] = T(s15);
      o[12 + d] = T(float(sd - double(s15)));
    } else {
      o[d] = T(sd);
      o[4 + d] = T(0);
      o[8 + d] = T(sd);
      o[12 + d] = T(0);
    }
    frc[4 * (size_t)n + d] = T(F[3 * (size_t)n + d]);
    const int cd = M > 0 ? (int)(sd * M) : 0;
    c[d] = cd < 0 ? 0 : (M > 0 && cd >= M ? M - 1 : cd);
  }
  o[3] = o[7] = o[11] = o[15] = T(0);
  frc[4 * (size_t)n + 3] = T(0);
  if (key != nullptr) {
    key[n] = (unsigned int)(c[0] + M * (c[1] + M * c[2]));
    idx[n] = n;
  }
}

// first and one-past-last sorted position of every cell (cells start empty: 0, 0)
__global__ void k_per_cell_bounds(int N, const unsigned int* __restrict__ skey, int* __restrict__ cstart,
                                  int* __restrict__ cend) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const unsigned int k = skey[i];
  if (i == 0 || skey[i - 1] != k) cstart[k] = i;
  if (i == N - 1 || skey[i + 1] != k) cend[k] = i + 1;
}

// u += t, compensated (Kahan) in FP32: the parts of the Ewald sum cancel to a small net
template <typename T> __device__ __forceinline__ void per_add(T& u, T& c, T t) {
  if constexpr (std::is_same<T, float>::value) {
    const T y = t - c;
    const T s = u + y;
    c = (s - u) - y;
    u = s;
  } else {
    u += t;
  }
}

template <typename T>
__device__ __forceinline__ void per_real_term(T dx, T dy, T dz, T rc2, T xi, const T* f, T* u, T* uc) {
  const T r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 < rc2)) return;
  const T r = sqrt(r2);
  const T xr = xi * r;
  const T e = per_exp(-xr * xr);
  const T c = T(2.0 / kSqrtPi) * xi;
  const T f1 = per_erfc(xr) - c * r * e;
  const T f2 = T(2) * c * (xr * xr - T(1)) * e;
  const T a = f2 + f1 / r;
  const T b = (f2 - f1 / r) / r2;
  const T dF = dx * f[0] + dy * f[1] + dz * f[2];
  per_add(u[0], uc[0], a * f[0] - b * dF * dx);
  per_add(u[1], uc[1], a * f[1] - b * dF * dy);
  per_add(u[2], uc[2], a * f[2] - b * dF * dz);
}

// real-space sum of target n: the sources of the 27 cells around its own (M >= 3), or
// every source (M = 0), by the minimum image
template <typename T>
__global__ void __launch_bounds__(kPerThreads) k_per_real(int N, double L, int M, double rc, double xi,
                                                          const T* __restrict__ pos, const T* __restrict__ frc,
                                                          const unsigned int* __restrict__ key,
                                                          const int* __restrict__ sidx, const int* __restrict__ cstart,
                                                          const int* __restrict__ cend, T* __restrict__ u_out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const T Lt = T(L), rc2 = T(rc * rc), xit = T(xi);
  const T* pn = pos + 16 * (size_t)n;
  T u[3] = {T(0), T(0), T(0)}, uc[3] = {T(0), T(0), T(0)};
  auto term = [&](int m) {
    if (m == n) return;
    const T* pm = pos + 16 * (size_t)m;
    T ds[3];
    for (int d = 0; d < 3; ++d) {
      T v = (pn[d] - pm[d]) + (pn[4 + d] - pm[4 + d]);   // cell units, exact wrap below
      v -= per_rint(v);
      ds[d] = v * Lt;
    }
    const T f[3] = {frc[4 * (size_t)m], frc[4 * (size_t)m + 1], frc[4 * (size_t)m + 2]};
    per_real_term<T>(ds[0], ds[1], ds[2], rc2, xit, f, u, uc);
  };
  if (M == 0) {
    for (int m = 0; m < N; ++m) term(m);
  } else {
    // the target's cell, as the sort saw it
    const unsigned int kn = key[n];
    const int c[3] = {(int)(kn % (unsigned)M), (int)((kn / (unsigned)M) % (unsigned)M), (int)(kn / ((unsigned)M * M))};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const int cx = (c[0] + ox + M) % M, cy = (c[1] + oy + M) % M, cz = (c[2] + oz + M) % M;
          const int cell = cx + M * (cy + M * cz);
          const int e = cend[cell];
          for (int i = cstart[cell]; i < e; ++i) term(sidx[i]);
        }
  }
  for (int d = 0; d < 3; ++d) u_out[3 * (size_t)n + d] = u[d];
}

// structure factors S(k) = sum_m F_m e^{-i k.R_m} (re, im of each component), one thread per k
template <typename T>
__global__ void __launch_bounds__(kPerThreads) k_per_struct(int N, long long nk, const T* __restrict__ kv,
                                                            const T* __restrict__ pos, const T* __restrict__ frc,
                                                            T* __restrict__ S) {
  __shared__ T sp[kPerTile * 8], sf[kPerTile * 4];
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = q < nk;
  T mx = T(0), my = T(0), mz = T(0);
  if (live) {
    mx = kv[4 * q];
    my = kv[4 * q + 1];
    mz = kv[4 * q + 2];
  }
  T re[3] = {T(0), T(0), T(0)}, im[3] = {T(0), T(0), T(0)};
  for (int base = 0; base < N; base += kPerTile) {
    const int len = min(kPerTile, N - base);
    __syncthreads();
    for (int i = threadIdx.x; i < len * 8; i += blockDim.x) sp[i] = pos[((size_t)base + i / 8) * 16 + 8 + i % 8];
    for (int i = threadIdx.x; i < len * 4; i += blockDim.x) sf[i] = frc[(size_t)base * 4 + i];
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < len; ++j) {
      // phase in cycles: frac(m.s15) + m.s_rem
      const T w = mx * sp[8 * j] + my * sp[8 * j + 1] + mz * sp[8 * j + 2];
      const T f = (w - per_floor(w)) + (mx * sp[8 * j + 4] + my * sp[8 * j + 5] + mz * sp[8 * j + 6]);
      T s, c;
      per_sincos2pi(f, &s, &c);
      for (int d = 0; d < 3; ++d) {
        re[d] += sf[4 * j + d] * c;
        im[d] -= sf[4 * j + d] * s;
      }
    }
  }
  if (!live) return;
  for (int d = 0; d < 3; ++d) {
    S[6 * q + d] = re[d];
    S[6 * q + 3 + d] = im[d];
  }
}

// wave-space sum of every target and the final velocities
template <typename T>
__global__ void __launch_bounds__(kPerThreads) k_per_recip(int N, long long nk, double xi, double a, double eta,
                                                           const T* __restrict__ kv, const T* __restrict__ S,
                                                           const T* __restrict__ pos, const T* __restrict__ frc,
                                                           const T* __restrict__ u_real, const double* __restrict__ Va,
                                                           double* __restrict__ V) {
  __shared__ T sk[kPerTile * 4], ss[kPerTile * 6];
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = n < N;
  T w15[3] = {T(0), T(0), T(0)}, wr[3] = {T(0), T(0), T(0)};
  if (live)
    for (int d = 0; d < 3; ++d) {
      w15[d] = pos[16 * (size_t)n + 8 + d];
      wr[d] = pos[16 * (size_t)n + 12 + d];
    }
  T u[3] = {T(0), T(0), T(0)}, uc[3] = {T(0), T(0), T(0)};
  for (long long base = 0; base < nk; base += kPerTile) {
    const int len = (int)min((long long)kPerTile, nk - base);
    __syncthreads();
    for (int i = threadIdx.x; i < len * 4; i += blockDim.x) sk[i] = kv[base * 4 + i];
    for (int i = threadIdx.x; i < len * 6; i += blockDim.x) ss[i] = S[base * 6 + i];
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < len; ++j) {
      const T kx = sk[4 * j], ky = sk[4 * j + 1], kz = sk[4 * j + 2], pref = sk[4 * j + 3];   // m and prefactor
      const T w = kx * w15[0] + ky * w15[1] + kz * w15[2];
      const T f = (w - per_floor(w)) + (kx * wr[0] + ky * wr[1] + kz * wr[2]);
      T s, c;
      per_sincos2pi(f, &s, &c);
      // w = Re[S e^{i k.R_n}], projected normal to k
      const T wx = ss[6 * j] * c - ss[6 * j + 3] * s;
      const T wy = ss[6 * j + 1] * c - ss[6 * j + 4] * s;
      const T wz = ss[6 * j + 2] * c - ss[6 * j + 5] * s;
      const T kw = (kx * wx + ky * wy + kz * wz) / (kx * kx + ky * ky + kz * kz);
      per_add(u[0], uc[0], pref * (wx - kw * kx));
      per_add(u[1], uc[1], pref * (wy - kw * ky));
      per_add(u[2], uc[2], pref * (wz - kw * kz));
    }
  }
  if (!live) return;
  const double self = 8.0 * xi / kSqrtPi;
  const double mob = 1.0 / (6.0 * kPi * eta * a), g = 1.0 / (8.0 * kPi * eta);
  for (int d = 0; d < 3; ++d) {
    const double f = double(frc[4 * (size_t)n + d]);
    const double un = double(u_real[3 * (size_t)n + d]) + double(u[d]) - self * f;
    V[3 * (size_t)n + d] = Va[3 * (size_t)n + d] + mob * f + g * un;
  }
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename T>
gbi_status run_periodic(gbi_ctx* ctx, int N, double L, double a, double eta, const double* R, const double* Va,
                        const double* Fe, double* V, const EwaldPlan& p) {
  std::vector<T> kv;
  ewald_kvectors<T>(p, L, kv);
  const long long nk = (long long)kv.size() / 4;
  const int M = p.M;
  const size_t ncell = M > 0 ? (size_t)M * M * M : 1;
  // temporary storage of the radix sort
  size_t sort_bytes = 0;
  if (M > 0)
    GBI_CHECK(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (const unsigned int*)nullptr, (unsigned int*)nullptr,
                                              (const int*)nullptr, (int*)nullptr, N, 0, 32, ctx->stream));
  const size_t o_pos = 0;
  const size_t o_frc = o_pos + al256(sizeof(T) * 16 * (size_t)N);
  const size_t o_ur = o_frc + al256(sizeof(T) * 4 * (size_t)N);
  const size_t o_kv = o_ur + al256(sizeof(T) * 3 * (size_t)N);
  const size_t o_S = o_kv + al256(sizeof(T) * 4 * (size_t)std::max(nk, 1ll));
  const size_t o_key = o_S + al256(sizeof(T) * 6 * (size_t)std::max(nk, 1ll));
  const size_t o_skey = o_key + al256(sizeof(unsigned int) * (size_t)N);
  const size_t o_idx = o_skey + al256(sizeof(unsigned int) * (size_t)N);
  const size_t o_sidx = o_idx + al256(sizeof(int) * (size_t)N);
  const size_t o_cs = o_sidx + al256(sizeof(int) * (size_t)N);
  const size_t o_ce = o_cs + al256(sizeof(int) * ncell);
  const size_t o_tmp = o_ce + al256(sizeof(int) * ncell);
  const size_t total = o_tmp + al256(sort_bytes + 1);
  GBI_TRY(ensure(ctx, ctx->perbuf, total));
  char* b = static_cast<char*>(ctx->perbuf.p);
  T* pos = reinterpret_cast<T*>(b + o_pos);
  T* frc = reinterpret_cast<T*>(b + o_frc);
  T* ur = reinterpret_cast<T*>(b + o_ur);
  T* kvd = reinterpret_cast<T*>(b + o_kv);
  T* S = reinterpret_cast<T*>(b + o_S);
  unsigned int* key = reinterpret_cast<unsigned int*>(b + o_key);
  unsigned int* skey = reinterpret_cast<unsigned int*>(b + o_skey);
  int* idx = reinterpret_cast<int*>(b + o_idx);
  int* sidx = reinterpret_cast<int*>(b + o_sidx);
  int* cs = reinterpret_cast<int*>(b + o_cs);
  int* ce = reinterpret_cast<int*>(b + o_ce);
  if (nk > 0) {
    GBI_CHECK(cudaMemcpyAsync(kvd, kv.data(), sizeof(T) * kv.size(), cudaMemcpyHostToDevice, ctx->stream));
  }
  k_per_records<T><<<grid1(N), 256, 0, ctx->stream>>>(N, L, M, R, Fe, pos, frc, M > 0 ? key : nullptr, idx);
  ++ctx->launches;
  if (M > 0) {
    size_t tb = sort_bytes;
    GBI_CHECK(cub::DeviceRadixSort::SortPairs(b + o_tmp, tb, key, skey, idx, sidx, N, 0, 32, ctx->stream));
    GBI_CHECK(cudaMemsetAsync(cs, 0, sizeof(int) * ncell, ctx->stream));
    GBI_CHECK(cudaMemsetAsync(ce, 0, sizeof(int) * ncell, ctx->stream));
    k_per_cell_bounds<<<grid1(N), 256, 0, ctx->stream>>>(N, skey, cs, ce);
    ctx->launches += 2;
  }
  k_per_real<T><<<grid1(N, kPerThreads), kPerThreads, 0, ctx->stream>>>(N, L, M, p.rc, p.xi, pos, frc, key, sidx, cs,
                                                                         ce, ur);
  k_per_struct<T><<<(unsigned)((std::max(nk, 1ll) + kPerThreads - 1) / kPerThreads), kPerThreads, 0, ctx->stream>>>(
      N, nk, kvd, pos, frc, S);
  k_per_recip<T><<<grid1(N, kPerThreads), kPerThreads, 0, ctx->stream>>>(N, nk, p.xi, a, eta, kvd, S, pos, frc, ur,
                                                                          Va, V);
  ctx->launches += 3;
  GBI_CHECK(cudaGetLastError());
  // the host copy of the wave vectors must outlive the transfer
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  return GBI_OK;
}

}  // namespace
}  // namespace gbi

using namespace gbi;

extern "C" gbi_status gbi_periodic_superpose(gbi_ctx* ctx, const gbi_params* prm, int N, double L, const double* R,
                                             const double* Va, const double* Fe, double* V, int* cells_per_side,
                                             double* xi, long long* n_wave) {
  if (!ctx || !valid_params(prm) || N < 0 || !(L > 0)) return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Fe || !V) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  const bool fp32 = prm->precision == 1 || prm->precision == 3;
  const EwaldPlan p = ewald_plan(N, L, fp32, cells_per_side ? *cells_per_side : 0);
  if (cells_per_side) *cells_per_side = p.M;
  if (xi) *xi = p.xi;
  if (n_wave) {
    std::vector<float> kv;
    ewald_kvectors<float>(p, L, kv);
    *n_wave = (long long)kv.size() / 4;
  }
  if (fp32) return run_periodic<float>(ctx, N, L, prm->a, prm->eta, R, Va, Fe, V, p);
  return run_periodic<double>(ctx, N, L, prm->a, prm->eta, R, Va, Fe, V, p);
}
