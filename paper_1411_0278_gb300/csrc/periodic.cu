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
//
// Particle-mesh form of the wave-space sum (smooth particle-mesh Ewald, Essmann et al.
// 1995): every force is spread onto a K^3 mesh with cardinal B-splines of order 8, the
// mesh is Fourier transformed (radix-2 kernels of this file; the x and y components
// packed as the real and imaginary parts of one complex grid, z in a second), each
// frequency multiplied by G^rec(k) |b(k)|^2 / L^3 (b the B-spline Fourier factors, k = 0
// left out), transformed back, and each sphere gathers its velocity with the same spline
// weights.  K >= 5 xi L keeps the mesh error near 1e-6 of the velocities.  Cost ~ N p^3 +
// K^3 log K instead of N n_k, and the real-space cut-off can shrink with the cells, so
// the whole sum grows as N log N.  The mesh is FP32 or FP64 with the sums.  Spreading
// adds with atomics, so the last bits of that part depend on timing.
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

// four doubles on a 32-byte boundary (the FP64 counterpart of float4)
struct alignas(32) Dbl4 {
  double x, y, z, w;
};

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

// the cell fraction s in [0, 1) of coordinate d of sphere n
__device__ __forceinline__ double per_frac(const double* __restrict__ R, size_t n, int d, double L) {
  double sd = R[3 * n + d] / L;
  sd -= floor(sd);                        // into [0, 1)
  if (!(sd < 1.0)) sd = 0.0;              // rounding up to 1
  return sd;
}

// the cell key of every sphere (cells c_d = floor(M s_d)) and the identity permutation
__global__ void k_per_keys(int N, double L, int M, const double* __restrict__ R, unsigned int* __restrict__ key,
                           int* __restrict__ idx) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int c[3];
  for (int d = 0; d < 3; ++d) {
    const int cd = (int)(per_frac(R, (size_t)n, d, L) * M);
    c[d] = cd < 0 ? 0 : (cd >= M ? M - 1 : cd);
  }
  key[n] = (unsigned int)(c[0] + M * (c[1] + M * c[2]));
  idx[n] = n;
}

// Record t (sphere n = order[t], or t without a sort): pos[16] = s_hi (3), 0, s_lo (3), 0,
// s15 (3), 0, s_rem (3), 0 of the cell fraction s (FP64: s, 0, s, 0); frc[4] = F, 0.
template <typename T>
__global__ void k_per_records(int N, double L, const double* __restrict__ R, const double* __restrict__ F,
                              const int* __restrict__ order, T* __restrict__ pos, T* __restrict__ frc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const size_t n = order ? (size_t)order[t] : (size_t)t;
  constexpr bool F32 = std::is_same<T, float>::value;
  T* o = pos + 16 * (size_t)t;
  for (int d = 0; d < 3; ++d) {
    const double sd = per_frac(R, n, d, L);
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
    frc[4 * (size_t)t + d] = T(F[3 * n + d]);
  }
  o[3] = o[7] = o[11] = o[15] = T(0);
  frc[4 * (size_t)t + 3] = T(0);
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
  T r, rinv;
  if constexpr (std::is_same<T, float>::value) {
    rinv = rsqrtf(r2);   // one reciprocal square root for r, 1/r and 1/r^2
    r = r2 * rinv;
  } else {
    r = sqrt(r2);
    rinv = T(1) / r;
  }
  const T xr = xi * r;
  const T e = per_exp(-xr * xr);
  const T c = T(2.0 / kSqrtPi) * xi;
  const T f1 = per_erfc(xr) - c * r * e;
  const T f2 = T(2) * c * (xr * xr - T(1)) * e;
  const T f1r = f1 * rinv;
  const T a = f2 + f1r;
  const T b = (f2 - f1r) * (rinv * rinv);
  const T dF = dx * f[0] + dy * f[1] + dz * f[2];
  per_add(u[0], uc[0], a * f[0] - b * dF * dx);
  per_add(u[1], uc[1], a * f[1] - b * dF * dy);
  per_add(u[2], uc[2], a * f[2] - b * dF * dz);
}

// Source records staged in shared memory: sp[8 j..] = s_hi, 0, s_lo, 0 and sf[4 j..] = F, 0 of
// records i0 .. i0 + len - 1.
template <typename T>
__device__ __forceinline__ void per_stage(const T* __restrict__ pos, const T* __restrict__ frc, int i0, int len,
                                          T* sp, T* sf) {
  for (int i = threadIdx.x; i < len * 8; i += blockDim.x) sp[i] = pos[16 * (size_t)(i0 + i / 8) + i % 8];
  for (int i = threadIdx.x; i < len * 4; i += blockDim.x) sf[i] = frc[4 * (size_t)i0 + i];
}

// separation (target - staged source j) by the minimum image, in length units, and its square
template <typename T>
__device__ __forceinline__ T per_sep(const T* pn, const T* sp, int j, T Lt, T* ds) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T v = (pn[d] - sp[8 * j + d]) + (pn[4 + d] - sp[8 * j + 4 + d]);   // cell units, exact wrap below
    v -= per_rint(v);
    ds[d] = v * Lt;
  }
  return ds[0] * ds[0] + ds[1] * ds[1] + ds[2] * ds[2];
}

// the real-space term of staged source j on a target with fractions pn (hi, 0, lo, 0)
template <typename T>
__device__ __forceinline__ void per_real_staged(const T* pn, const T* sp, const T* sf, int j, T Lt, T rc2, T xit,
                                                T* u, T* uc) {
  T ds[3];
  per_sep<T>(pn, sp, j, Lt, ds);
  const T f[3] = {sf[4 * j], sf[4 * j + 1], sf[4 * j + 2]};
  per_real_term<T>(ds[0], ds[1], ds[2], rc2, xit, f, u, uc);
}

// Real-space sums by cells (M >= 3, records in cell order).  blockIdx.x is the target
// cell, blockIdx.y one of gridDim.y passes over its records, kPerCellSlots targets per pass.
// The sources of the 27 cells around it (ranges of the cell order) are staged in shared
// memory in chunks of up to kPerCellCap records; thread (slot, quarter) adds to target
// `slot` the chunk's sources j = quarter (mod 4).  Sources are taken 32 at a time: first a
// bit mask of those within the cut-off (r > 0 leaves the target itself out), then only
// those are evaluated, so the lanes of a warp diverge only in how many.  The four quarters'
// compensated sums are added at the end.
constexpr int kPerCellThreads = 256;
constexpr int kPerCellSlots = 64;
constexpr int kPerCellQuarters = kPerCellThreads / kPerCellSlots;
template <typename T> struct PerCellCap { static constexpr int v = sizeof(T) == 4 ? 1024 : 512; };

template <typename T> struct PerQuad;
template <> struct PerQuad<float> { using t = float4; };
template <> struct PerQuad<double> { using t = Dbl4; };

template <typename T>
__global__ void __launch_bounds__(kPerCellThreads)
    k_per_real_cells(int M, double L, double rc, double xi, const T* __restrict__ pos, const T* __restrict__ frc,
                     const int* __restrict__ cstart, const int* __restrict__ cend, T* __restrict__ u_out) {
  using Q4 = typename PerQuad<T>::t;
  constexpr int kCap = PerCellCap<T>::v;
  // source j: sa = (s_hi, F_x), sb = (s_lo, F_y), sc = F_z
  __shared__ Q4 sa[kCap], sb[kCap];
  __shared__ T sc[kCap];
  __shared__ int r_start[27], r_pre[28];
  __shared__ T red[kPerCellQuarters - 1][kPerCellSlots][3];
  const int cell = blockIdx.x;
  const int c[3] = {cell % M, (cell / M) % M, cell / (M * M)};
  const int t0 = cstart[cell], t1 = cend[cell];
  if (threadIdx.x < 27) {
    const int o = threadIdx.x;
    const int cx = (c[0] + o % 3 - 1 + M) % M, cy = (c[1] + (o / 3) % 3 - 1 + M) % M,
              cz = (c[2] + o / 9 - 1 + M) % M;
    const int nb = cx + M * (cy + M * cz);
    r_start[o] = cstart[nb];
    r_pre[o + 1] = cend[nb] - cstart[nb];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    r_pre[0] = 0;
    for (int o = 0; o < 27; ++o) r_pre[o + 1] += r_pre[o];
  }
  __syncthreads();
  const int total = r_pre[27];
  const int slot = threadIdx.x % kPerCellSlots, quarter = threadIdx.x / kPerCellSlots;
  const T Lt = T(L), rc2 = T(rc * rc), xit = T(xi);
  for (int tp = t0 + blockIdx.y * kPerCellSlots; tp < t1; tp += gridDim.y * kPerCellSlots) {
    const int t = tp + slot;
    const bool live = t < t1;
    T pn[8];
    {
      const int tl = live ? t : t0;
#pragma unroll
      for (int j = 0; j < 8; ++j) pn[j] = pos[16 * (size_t)tl + j];
    }
    T u[3] = {T(0), T(0), T(0)}, uc[3] = {T(0), T(0), T(0)};
    for (int base = 0; base < total; base += kCap) {
      const int n = min(kCap, total - base);
      __syncthreads();   // the previous chunk is done
      // stage records base .. base + n - 1 of the 27 ranges (loads issued together)
      constexpr int kPer = kCap / kPerCellThreads;
      Q4 la[kPer], lb[kPer];
      T lc[kPer];
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int e = threadIdx.x + k * kPerCellThreads;
        if (e < n) {
          const int g = base + e;
          int o = 0;
          while (o < 26 && r_pre[o + 1] <= g) ++o;
          const size_t m = (size_t)(r_start[o] + (g - r_pre[o]));
          const T* pm = pos + 16 * m;
          const T* fm = frc + 4 * m;
          la[k] = Q4{pm[0], pm[1], pm[2], fm[0]};
          lb[k] = Q4{pm[4], pm[5], pm[6], fm[1]};
          lc[k] = fm[2];
        }
      }
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int e = threadIdx.x + k * kPerCellThreads;
        if (e < n) {
          sa[e] = la[k];
          sb[e] = lb[k];
          sc[e] = lc[k];
        }
      }
      __syncthreads();
      if (!live) continue;
      const int ni = (n - quarter + kPerCellQuarters - 1) / kPerCellQuarters;   // j = quarter + 4 i
      for (int ib = 0; ib < ni; ib += 32) {
        unsigned int mask = 0u;
        // the cut-off test on the high parts alone (a pair it misjudges sits at r_c, where
        // its term is erfc(xi r_c) ~ 3e-9 of a near pair's); the target itself gives r2 = 0
#pragma unroll
        for (int bit = 0; bit < 32; ++bit) {
          const int i = ib + bit;
          if (i < ni) {
            const int j = quarter + kPerCellQuarters * i;
            const Q4 qa = sa[j];
            T v0 = pn[0] - qa.x, v1 = pn[1] - qa.y, v2 = pn[2] - qa.z;
            v0 = (v0 - per_rint(v0)) * Lt;
            v1 = (v1 - per_rint(v1)) * Lt;
            v2 = (v2 - per_rint(v2)) * Lt;
            const T r2 = v0 * v0 + v1 * v1 + v2 * v2;
            mask |= (r2 < rc2 && r2 > T(0) ? 1u : 0u) << bit;
          }
        }
        while (mask) {
          const int bit = __ffs(mask) - 1;
          mask &= mask - 1u;
          const int j = quarter + kPerCellQuarters * (ib + bit);
          const Q4 qa = sa[j], qb = sb[j];
          T v0 = (pn[0] - qa.x) + (pn[4] - qb.x), v1 = (pn[1] - qa.y) + (pn[5] - qb.y),
            v2 = (pn[2] - qa.z) + (pn[6] - qb.z);
          v0 = (v0 - per_rint(v0)) * Lt;
          v1 = (v1 - per_rint(v1)) * Lt;
          v2 = (v2 - per_rint(v2)) * Lt;
          const T f[3] = {qa.w, qb.w, sc[j]};
          per_real_term<T>(v0, v1, v2, rc2, xit, f, u, uc);
        }
      }
    }
    // the quarters' sums: quarters 1..3 hand theirs to quarter 0
    __syncthreads();
    if (quarter > 0 && live)
      for (int d = 0; d < 3; ++d) red[quarter - 1][slot][d] = u[d] - uc[d];
    __syncthreads();
    if (quarter == 0 && live) {
      for (int d = 0; d < 3; ++d) {
        T acc = u[d] - uc[d];
        for (int q = 0; q < kPerCellQuarters - 1; ++q) acc += red[q][slot][d];
        u_out[3 * (size_t)t + d] = acc;
      }
    }
  }
}

// Real-space sums over every pair by the minimum image (rc = L / 2): one thread per target
// record, sources staged in shared memory in tiles.
template <typename T>
__global__ void __launch_bounds__(kPerThreads) k_per_real_all(int N, double L, double rc, double xi,
                                                              const T* __restrict__ pos, const T* __restrict__ frc,
                                                              T* __restrict__ u_out) {
  __shared__ T sp[kPerTile * 8], sf[kPerTile * 4];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = t < N;
  const T Lt = T(L), rc2 = T(rc * rc), xit = T(xi);
  T pn[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) pn[j] = live ? pos[16 * (size_t)t + j] : T(0);
  T u[3] = {T(0), T(0), T(0)}, uc[3] = {T(0), T(0), T(0)};
  for (int sb = 0; sb < N; sb += kPerTile) {
    const int len = min(kPerTile, N - sb);
    __syncthreads();
    per_stage<T>(pos, frc, sb, len, sp, sf);
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < len; ++j)
      if (sb + j != t) per_real_staged<T>(pn, sp, sf, j, Lt, rc2, xit, u, uc);
  }
  if (live)
    for (int d = 0; d < 3; ++d) u_out[3 * (size_t)t + d] = u[d];
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

// wave-space sum of every target record and the final velocities
template <typename T>
__global__ void __launch_bounds__(kPerThreads) k_per_recip(int N, long long nk, double xi, double a, double eta,
                                                           const T* __restrict__ kv, const T* __restrict__ S,
                                                           const T* __restrict__ pos, const int* __restrict__ order,
                                                           const double* __restrict__ Fe,
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
  // record n is sphere order[n]
  const size_t sn = order ? (size_t)order[n] : (size_t)n;
  const double self = 8.0 * xi / kSqrtPi;
  const double mob = 1.0 / (6.0 * kPi * eta * a), g = 1.0 / (8.0 * kPi * eta);
  for (int d = 0; d < 3; ++d) {
    const double f = Fe[3 * sn + d];
    const double un = double(u_real[3 * (size_t)n + d]) + double(u[d]) - self * f;
    V[3 * sn + d] = Va[3 * sn + d] + mob * f + g * un;
  }
}

// ---------------------------------------------------------------------------------
// particle mesh
// ---------------------------------------------------------------------------------
constexpr int kPmeOrder = 8;        // cardinal B-splines of order 8 (degree 7)
constexpr double kPmeMeshPerXiL = 5.0;   // K >= 5 xi L keeps the mesh error near 1e-6 of the velocities
constexpr int kPmeFftThreads = 256;

// complex values of the mesh and the staging points (x, y, z, unused) that spreading adds into
template <typename G> struct Cplx;
template <> struct Cplx<float> {
  using t = float2;
  using q = float4;
};
template <> struct Cplx<double> {
  using t = double2;
  using q = Dbl4;
};

// weights w[j] = M_p(f + j), j = 0..p-1, of the grid points floor(u) - j (cardinal
// B-spline M_p on [0, p], f the fraction of u), by the recursion
// M_n(x) = (x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)) / (n - 1) from M_2(x) = 1 - |x - 1|
template <typename G> __device__ __forceinline__ void pme_weights(G f, G* w) {
  w[0] = f;
  w[1] = G(1) - f;
#pragma unroll
  for (int j = 2; j < kPmeOrder; ++j) w[j] = G(0);
#pragma unroll
  for (int n = 3; n <= kPmeOrder; ++n) {
    const G inv = G(1) / G(n - 1);
#pragma unroll
    for (int j = n - 1; j >= 0; --j) {
      const G x = f + G(j);
      const G prev = j > 0 ? w[j - 1] : G(0);
      w[j] = (x * w[j] + (G(n) - x) * prev) * inv;
    }
  }
}

// grid coordinate u = K s of a position (s the cell fraction in [0, 1)): first point k0
// (the points are k0 - j mod K) and the spline weights of each axis
template <typename G>
__device__ __forceinline__ void pme_point(const double* __restrict__ R, size_t n, double L, int K, int* k0,
                                          G (*w)[kPmeOrder]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double s = R[3 * n + d] / L;
    s -= floor(s);
    if (!(s < 1.0)) s = 0.0;
    const double u = s * K;
    const double fl = floor(u);
    k0[d] = (int)fl;
    pme_weights<G>(G(u - fl), w[d]);
  }
}

__device__ __forceinline__ int pme_wrap(int g, int K) { return g < 0 ? g + K : g; }   // g > -K

// Spreading, in the order of the cell sort (neighbouring threads touch neighbouring
// points): Q(g) = sum_n F_n w_n(g) over the p^3 points of every sphere, the three
// components of a point added together (one vector atomic in FP32)
__device__ __forceinline__ void pme_add(float4* q, float wx, float wy, float wz) {
  atomicAdd(q, make_float4(wx, wy, wz, 0.0f));
}
__device__ __forceinline__ void pme_add(Dbl4* q, double wx, double wy, double wz) {
  atomicAdd(&q->x, wx);
  atomicAdd(&q->y, wy);
  atomicAdd(&q->z, wz);
}

// eight lanes per sphere, lane jx taking the grid points k0_x - jx (a warp's accesses are
// runs of eight neighbouring points)
constexpr int kPmeLanes = kPmeOrder;

template <typename G>
__global__ void k_pme_spread(int N, int K, const double* __restrict__ R, double L, const double* __restrict__ F,
                             const int* __restrict__ order, typename Cplx<G>::q* __restrict__ Q) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt / kPmeLanes), jx = (int)(gt % kPmeLanes);
  if (t >= N) return;
  const int n = order[t];
  int k0[3];
  G w[3][kPmeOrder];
  pme_point<G>(R, (size_t)n, L, K, k0, w);
  G wx = w[0][0];
#pragma unroll
  for (int j = 1; j < kPmeOrder; ++j)
    if (j == jx) wx = w[0][j];
  const G Fx = G(F[3 * (size_t)n]) * wx, Fy = G(F[3 * (size_t)n + 1]) * wx, Fz = G(F[3 * (size_t)n + 2]) * wx;
  const size_t gx = (size_t)pme_wrap(k0[0] - jx, K);
#pragma unroll
  for (int jz = 0; jz < kPmeOrder; ++jz) {
    const size_t gz = (size_t)pme_wrap(k0[2] - jz, K);
#pragma unroll
    for (int jy = 0; jy < kPmeOrder; ++jy) {
      const size_t row = (size_t)K * ((size_t)pme_wrap(k0[1] - jy, K) + (size_t)K * gz);
      const G wyz = w[1][jy] * w[2][jz];
      pme_add(&Q[row + gx], wyz * Fx, wyz * Fy, wyz * Fz);
    }
  }
}

// the most elements (LB K) an FFT block holds
template <typename G> __host__ __device__ constexpr int pme_max_line_elems() { return sizeof(G) == 4 ? 4096 : 2048; }

// ---- line FFT: four steps (K = 16 N2, N2 in {1, 2, 4, 8, 16, 32}) --------------------
//
// x[N2 n1 + n2] -> X[k1 + 16 k2] = sum_n2 e^{-+2 pi i n2 k2 / N2} [e^{-+2 pi i n2 k1 / K}
// sum_n1 x[N2 n1 + n2] e^{-+2 pi i n1 k1 / 16}]: a 16-point DFT per n2 in registers (reading
// and writing the same 16 elements, so no barrier), the twiddles, then an N2-point DFT per
// k1 in registers.  Rows are padded by one element after every 16 (pme_pad) so that both
// the strided and the contiguous register loads avoid bank conflicts.

// e^{2 pi i k / 32}: cos and sin of k pi / 16, k = 0..15
__device__ __forceinline__ constexpr double pme_c32(int k) {
  constexpr double c[16] = {1.0,
                            0.98078528040323043,
                            0.92387953251128674,
                            0.83146961230254524,
                            0.70710678118654752,
                            0.55557023301960218,
                            0.38268343236508977,
                            0.19509032201612826,
                            0.0,
                            -0.19509032201612826,
                            -0.38268343236508977,
                            -0.55557023301960218,
                            -0.70710678118654752,
                            -0.83146961230254524,
                            -0.92387953251128674,
                            -0.98078528040323043};
  return c[k];
}
__device__ __forceinline__ constexpr double pme_s32(int k) { return pme_c32(k >= 8 ? k - 8 : 8 - k); }

__host__ __device__ constexpr int pme_log2(int n) { return n <= 1 ? 0 : 1 + pme_log2(n >> 1); }

// In-register DFT of N (<= 32) values, natural order in and out, e^{-2 pi i j k / N}
// (forward) or e^{+2 pi i j k / N} (INV): radix-2 Stockham passes between two register
// arrays (no permutation), every index a compile-time constant after unrolling.  With Ns
// the length done so far, butterfly j takes a[j] and a[j + N/2] e^{-+2 pi i k / (2 Ns)},
// k = j mod Ns, and writes outputs (j - k) 2 + k and that + Ns.
template <typename C, int N, bool INV>
__device__ __forceinline__ void pme_reg_fft(C* v) {
  using G = decltype(v[0].x);
  if constexpr (N > 1) {
    C a[N], b[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = v[i];
#pragma unroll
    for (int Ns = 1; Ns < N; Ns <<= 1) {
#pragma unroll
      for (int j = 0; j < N / 2; ++j) {
        const int k = j & (Ns - 1);
        const int t = k * (16 / Ns);   // e^{-+2 pi i k / (2 Ns)} = e^{-+2 pi i t / 32}
        const G wc = G(pme_c32(t)), ws = INV ? G(pme_s32(t)) : G(-pme_s32(t));
        const C x0 = a[j], y = a[j + N / 2];
        const G x1r = wc * y.x - ws * y.y, x1i = wc * y.y + ws * y.x;
        const int o = (j - k) * 2 + k;
        b[o] = C{x0.x + x1r, x0.y + x1i};
        b[o + Ns] = C{x0.x - x1r, x0.y - x1i};
      }
#pragma unroll
      for (int i = 0; i < N; ++i) a[i] = b[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = a[i];
  }
}

__host__ __device__ constexpr int pme_pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int pme_row(int K) { return K + K / 16 + 1; }

// The four-step transform of LB padded rows of K = 16 N2 values in shared memory (twf the
// K twiddles e^{-+2 pi i t / K}, conjugated for the inverse); barriers inside.
template <typename G, int N2, bool INV>
__device__ __forceinline__ void pme_fft4_rows(typename Cplx<G>::t* sx, const typename Cplx<G>::t* twf, int LB) {
  using C = typename Cplx<G>::t;
  constexpr int K = 16 * N2, RS = pme_row(K);
  // stage 1: task (row, n2)
  for (int task = threadIdx.x; task < LB * N2; task += blockDim.x) {
    const int lane = task / N2, n2 = task - lane * N2;
    C* row = sx + lane * RS;
    C v[16];
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) v[n1] = row[pme_pad(N2 * n1 + n2)];
    pme_reg_fft<C, 16, INV>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) {
      const C w = twf[n2 * k1];
      const C a = v[k1];
      v[k1] = C{w.x * a.x - w.y * a.y, w.x * a.y + w.y * a.x};
    }
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) row[pme_pad(N2 * k1 + n2)] = v[k1];
  }
  __syncthreads();
  // stage 2: task (row, k1), read everything before anything is written
  constexpr int kT = (16 * 4096 / K + kPmeFftThreads - 1) / kPmeFftThreads;   // tasks per thread at most
  C u[kT][N2];
#pragma unroll
  for (int t = 0; t < kT; ++t) {
    const int task = threadIdx.x + t * kPmeFftThreads;
    if (task < LB * 16) {
      const int lane = task >> 4, k1 = task & 15;
      const C* row = sx + lane * RS;
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) u[t][n2] = row[pme_pad(N2 * k1 + n2)];
      pme_reg_fft<C, N2, INV>(u[t]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < kT; ++t) {
    const int task = threadIdx.x + t * kPmeFftThreads;
    if (task < LB * 16) {
      const int lane = task >> 4, k1 = task & 15;
      C* row = sx + lane * RS;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) row[pme_pad(k1 + 16 * k2)] = u[t][k2];
    }
  }
  __syncthreads();
}

// In-place FFT of the K-point lines of one axis (K = 16 N2 <= 512), unnormalised,
// e^{-2 pi i m g / K} (forward) or e^{+2 pi i m g / K} (inverse), natural order in and out.
// The K^2 lines of a grid are numbered l = a + K b over the two other axes; line l holds
//   axis 0: K l + i,   axis 1: a + K^2 b + K i,   axis 2: l + K^2 i   (i = 0..K-1).
// A block transforms LB = 2^logLB consecutive lines (LB | K, LB K <= 4096 in FP32, 2048 in
// FP64) in shared memory; consecutive lines are adjacent in memory along axes 1 and 2, so
// those loads coalesce in runs of LB elements.  grids = A (blockIdx.y = 0) and B (1); with
// src the lines are read from the staging points instead (A = x + i y, B = z).
// tw[t] = e^{-2 pi i t / K}, t < K.  Indices are 32-bit (K^3 <= 2^27).
template <typename G, int N2>
__global__ void __launch_bounds__(kPmeFftThreads, (sizeof(G) == 4 && N2 >= 16) ? 3 : 1)
    k_pme_fft4(typename Cplx<G>::t* __restrict__ grids, const typename Cplx<G>::q* __restrict__ src, int logLB,
               int axis, int inverse, const typename Cplx<G>::t* __restrict__ tw) {
  using C = typename Cplx<G>::t;
  constexpr int K = 16 * N2, RS = pme_row(K), logK = pme_log2(K);
  extern __shared__ __align__(16) unsigned char pme_smem[];
  C* sx = reinterpret_cast<C*>(pme_smem);
  const int LB = 1 << logLB;
  C* stw = sx + (size_t)LB * RS;
  const unsigned int K2 = (unsigned)K * K;
  C* g = grids + (size_t)blockIdx.y * K2 * K;
  const unsigned int l0 = blockIdx.x << logLB;
  const unsigned int tot = (unsigned)LB * K;
  for (unsigned int j = threadIdx.x; j < (unsigned)K; j += blockDim.x) {
    C w = tw[j];
    if (inverse) w.y = -w.y;
    stw[j] = w;
  }
  auto at = [&](unsigned int e, unsigned int& si) -> unsigned int {
    unsigned int lane, i;
    if (axis == 0) {
      lane = e >> logK;
      i = e & (K - 1u);
      si = lane * RS + pme_pad((int)i);
      return ((l0 + lane) << logK) + i;
    }
    lane = e & ((unsigned)LB - 1u);
    i = e >> logLB;
    si = lane * RS + pme_pad((int)i);
    const unsigned int l = l0 + lane;
    if (axis == 1) return (l & (K - 1u)) + ((l >> logK) << (2 * logK)) + (i << logK);
    return l + (i << (2 * logK));
  };
  constexpr int kMaxE = pme_max_line_elems<G>() / kPmeFftThreads;
  C v[kMaxE];
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) {
      unsigned int si;
      const unsigned int ad = at(e, si);
      if (src) {
        const typename Cplx<G>::q q = src[ad];
        v[k] = blockIdx.y == 0 ? C{q.x, q.y} : C{q.z, G(0)};
      } else {
        v[k] = g[ad];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) {
      unsigned int si;
      at(e, si);
      sx[si] = v[k];
    }
  }
  __syncthreads();
  if (inverse)
    pme_fft4_rows<G, N2, true>(sx, stw, LB);
  else
    pme_fft4_rows<G, N2, false>(sx, stw, LB);
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) {
      unsigned int si;
      const unsigned int ad = at(e, si);
      g[ad] = sx[si];
    }
  }
}

// Wave space on the mesh, fused with the transforms along x.  On entry A = FT_yz(Q_x + i Q_y)
// and B = FT_yz(Q_z) (transformed along z and y); rows are the x-lines (y, z), K = 2^logK
// contiguous values each.  A block takes P = 2^logP consecutive rows (same z) and, for each
// row that owns its pair (row (y, z) and its mirror ((K - y) mod K, (K - z) mod K) with the
// row not above its mirror; a row that is its own mirror pairs with itself), loads the row
// and its mirror row of A and of B: 4P rows in shared memory.  It transforms them along x
// (now A = FT(Q_x + i Q_y), B = FT(Q_z) for those rows, natural order: index i holds
// m = i for i < K/2 and i - K otherwise), and at every frequency m forms
//   Q_x^(m) = (A(m) + conj A(-m)) / 2,  Q_y^(m) = (A(m) - conj A(-m)) / (2 i),  Q_z^(m) = B(m),
//   U(m) = T(m) Q^(m),  T(m) = G^rec(k_m) |b(m)|^2 / L^3
//        = 8 pi (I - k k / k^2) / k^2 (1 + q + 2 q^2) e^{-q} |b|^2 / L^3  (T(0) = 0: zero mean flow),
// A(m) = U_x + i U_y, B(m) = U_z (the mirror -m lies in the mirror row at (K - i) mod K), then
// transforms back along x and stores the rows it owns.  bmod[i] = |b_i|^2 of one axis.
template <typename G, int N2>
__global__ void __launch_bounds__(kPmeFftThreads)
    k_pme_xconv(typename Cplx<G>::t* __restrict__ A, typename Cplx<G>::t* __restrict__ B, int logP, double L,
                double xi, const G* __restrict__ bmod, const typename Cplx<G>::t* __restrict__ tw) {
  using C = typename Cplx<G>::t;
  extern __shared__ __align__(16) unsigned char pme_smem[];
  constexpr int RS = pme_row(16 * N2), logK = pme_log2(16 * N2);
  const unsigned int K = 16u * N2, mask = K - 1u, P = 1u << logP;
  const int logLB = logP + 2;   // rows: A own, A mirror, B own, B mirror
  const int LB = 1 << logLB;
  C* sx = reinterpret_cast<C*>(pme_smem);
  C* stw = sx + (size_t)LB * RS;
  const unsigned int r0 = blockIdx.x << logP;
  const unsigned int z = r0 >> logK, nz = (K - z) & mask;
  if (nz < z) return;   // the whole block's rows are mirrors of rows done elsewhere
  // row slot s: own row r0 + s, active unless its mirror is the lower row
  auto own_row = [&](unsigned int sl) { return r0 + sl; };
  auto mir_row = [&](unsigned int sl) {
    const unsigned int y = (r0 + sl) & mask;
    return ((K - y) & mask) + (nz << logK);
  };
  auto active = [&](unsigned int sl) { return own_row(sl) <= mir_row(sl); };
  // shared row q -> global element base
  auto row_base = [&](unsigned int q) -> C* {
    const unsigned int sl = q & (P - 1u);
    const bool mir = ((q >> logP) & 1u) != 0u;
    C* g = q < 2u * P ? A : B;
    return g + ((size_t)(mir ? mir_row(sl) : own_row(sl)) << logK);
  };
  for (unsigned int j = threadIdx.x; j < K; j += blockDim.x) stw[j] = tw[j];
  const unsigned int tot = 1u << (logLB + logK);
  constexpr int kMaxE = pme_max_line_elems<G>() / kPmeFftThreads;
  C v[kMaxE];
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) v[k] = row_base(e >> logK)[e & mask];
  }
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) sx[(e >> logK) * RS + pme_pad((int)(e & mask))] = v[k];
  }
  __syncthreads();
  pme_fft4_rows<G, N2, false>(sx, stw, LB);
  // the products: element e of the A rows (own and mirror) and the same element of B
  const G s = G(2.0 * kPi / L);
  const G c0 = G(8.0 * kPi / (L * L * L)), cq = G(0.25 / (xi * xi));
  const unsigned int ntot = 1u << (logP + 1 + logK);   // A own and mirror rows
  C ua[kMaxE / 2], ub[kMaxE / 2];
#pragma unroll
  for (int k = 0; k < kMaxE / 2; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < ntot) {
      const unsigned int q = e >> logK, ix = e & mask;
      const unsigned int sl = q & (P - 1u);
      const bool mir = q >= P;
      const unsigned int row = mir ? mir_row(sl) : own_row(sl);
      const unsigned int iy = row & mask, iz = row >> logK;
      const unsigned int qm = mir ? sl : sl + P;   // the paired row in shared memory
      const unsigned int nx = (K - ix) & mask;
      const C a = sx[q * RS + pme_pad((int)ix)], an = sx[qm * RS + pme_pad((int)nx)],
              b = sx[(q + 2u * P) * RS + pme_pad((int)ix)];
      if (row == 0u && ix == 0u) {
        ua[k] = C{G(0), G(0)};
        ub[k] = C{G(0), G(0)};
        continue;
      }
      const G qx_r = G(0.5) * (a.x + an.x), qx_i = G(0.5) * (a.y - an.y);
      const G qy_r = G(0.5) * (a.y + an.y), qy_i = G(0.5) * (an.x - a.x);
      const G qz_r = b.x, qz_i = b.y;
      const int mx = (int)ix < (int)K / 2 ? (int)ix : (int)ix - (int)K;
      const int my = (int)iy < (int)K / 2 ? (int)iy : (int)iy - (int)K;
      const int mz = (int)iz < (int)K / 2 ? (int)iz : (int)iz - (int)K;
      const G kx = s * G(mx), ky = s * G(my), kz = s * G(mz);
      const G k2 = kx * kx + ky * ky + kz * kz;
      const G ik2 = G(1) / k2;
      const G qq = k2 * cq;
      const G pref = c0 * ik2 * (G(1) + qq + G(2) * qq * qq) * per_exp(-qq) * bmod[ix] * bmod[iy] * bmod[iz];
      const G dr = (kx * qx_r + ky * qy_r + kz * qz_r) * ik2, di = (kx * qx_i + ky * qy_i + kz * qz_i) * ik2;
      const G ux_r = pref * (qx_r - kx * dr), ux_i = pref * (qx_i - kx * di);
      const G uy_r = pref * (qy_r - ky * dr), uy_i = pref * (qy_i - ky * di);
      const G uz_r = pref * (qz_r - kz * dr), uz_i = pref * (qz_i - kz * di);
      ua[k] = C{ux_r - uy_i, ux_i + uy_r};
      ub[k] = C{uz_r, uz_i};
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kMaxE / 2; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < ntot) {
      const unsigned int q = e >> logK, ix = e & mask;
      sx[q * RS + pme_pad((int)ix)] = ua[k];
      sx[(q + 2u * P) * RS + pme_pad((int)ix)] = ub[k];
    }
  }
  __syncthreads();
  for (unsigned int j = threadIdx.x; j < K; j += blockDim.x) stw[j].y = -stw[j].y;   // the inverse's twiddles
  __syncthreads();
  pme_fft4_rows<G, N2, true>(sx, stw, LB);
  // store the rows this block owns: own rows of active slots, mirror rows of active slots
  // that are not their own mirror
#pragma unroll
  for (int k = 0; k < kMaxE; ++k) {
    const unsigned int e = threadIdx.x + k * kPmeFftThreads;
    if (e < tot) {
      const unsigned int q = e >> logK;
      const unsigned int sl = q & (P - 1u);
      const bool mir = ((q >> logP) & 1u) != 0u;
      if (active(sl) && !(mir && mir_row(sl) == own_row(sl)))
        row_base(q)[e & mask] = sx[q * RS + pme_pad((int)(e & mask))];
    }
  }
}

// Gathering: the wave-space velocity of every sphere with its spline weights (u_x, u_y the
// real and imaginary parts of A, u_z the real part of B), and the final velocities
// V = Va + F / (6 pi eta a) + (u_real + u_wave - 8 xi / sqrt(pi) F) / (8 pi eta)
template <typename G, typename T>
__global__ void k_pme_gather(int N, int K, const double* __restrict__ R, double L, const double* __restrict__ F,
                             const int* __restrict__ order, const typename Cplx<G>::t* __restrict__ A,
                             const typename Cplx<G>::t* __restrict__ B, double xi, double a, double eta,
                             const T* __restrict__ u_real, const double* __restrict__ Va, double* __restrict__ V) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt / kPmeLanes), jx = (int)(gt % kPmeLanes);
  const bool live = t < N;   // the eight lanes of a sphere are live or not together
  const int n = live ? order[t] : 0;
  G u[3] = {G(0), G(0), G(0)}, uc[3] = {G(0), G(0), G(0)};
  if (live) {
    int k0[3];
    G w[3][kPmeOrder];
    pme_point<G>(R, (size_t)n, L, K, k0, w);
    G wx = w[0][0];
#pragma unroll
    for (int j = 1; j < kPmeOrder; ++j)
      if (j == jx) wx = w[0][j];
    const size_t gx = (size_t)pme_wrap(k0[0] - jx, K);
#pragma unroll
    for (int jz = 0; jz < kPmeOrder; ++jz) {
      const size_t gz = (size_t)pme_wrap(k0[2] - jz, K);
#pragma unroll
      for (int jy = 0; jy < kPmeOrder; ++jy) {
        const size_t g = (size_t)K * ((size_t)pme_wrap(k0[1] - jy, K) + (size_t)K * gz) + gx;
        const G ww = wx * w[1][jy] * w[2][jz];
        const typename Cplx<G>::t av = A[g];
        per_add(u[0], uc[0], ww * av.x);
        per_add(u[1], uc[1], ww * av.y);
        per_add(u[2], uc[2], ww * B[g].x);
      }
    }
  }
  // the eight lanes' partial sums (aligned groups of eight lanes of the warp)
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    u[d] -= uc[d];
#pragma unroll
    for (int off = kPmeLanes / 2; off > 0; off >>= 1) u[d] += __shfl_xor_sync(0xffffffffu, u[d], off);
  }
  if (!live || jx != 0) return;
  const double self = 8.0 * xi / kSqrtPi;
  const double mob = 1.0 / (6.0 * kPi * eta * a), gg = 1.0 / (8.0 * kPi * eta);
  for (int d = 0; d < 3; ++d) {
    const double f = F[3 * (size_t)n + d];
    const double un = double(u_real[3 * (size_t)t + d]) + double(u[d]) - self * f;   // record t
    V[3 * (size_t)n + d] = Va[3 * (size_t)n + d] + mob * f + gg * un;
  }
}

// |b(m)|^2 = 1 / |sum_{j=0}^{p-2} M_p(j + 1) e^{2 pi i m j / K}|^2 for m = 0..K-1 (the
// B-spline Fourier factors of smooth particle-mesh Ewald; p even, so no zero divisor)
std::vector<double> pme_bmod(int K) {
  // M_p at the integers 0..p-1, by the recursion above at f = 0
  double w[kPmeOrder];
  w[0] = 0.0;
  w[1] = 1.0;
  for (int j = 2; j < kPmeOrder; ++j) w[j] = 0.0;
  for (int n = 3; n <= kPmeOrder; ++n)
    for (int j = n - 1; j >= 0; --j) {
      const double prev = j > 0 ? w[j - 1] : 0.0;
      w[j] = (j * w[j] + (n - j) * prev) / (n - 1);
    }
  std::vector<double> out(K);
  for (int m = 0; m < K; ++m) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j <= kPmeOrder - 2; ++j) {
      const double arg = 2.0 * kPi * double(m) * j / K;
      re += w[j + 1] * std::cos(arg);
      im += w[j + 1] * std::sin(arg);
    }
    out[m] = 1.0 / (re * re + im * im);
  }
  return out;
}

// lines per FFT block: at most 36 KB of padded rows (plus K twiddles), at most 32, at least
// 4 (the fused x kernel's row quartets), dividing K, LB K within the elements a block holds
int pme_lines_per_block(int K, size_t elem) {
  const int cap = elem == sizeof(float2) ? 4096 : 2048;
  int lb = 1;
  while (lb < 32 && lb * 2 <= K && (size_t)(lb * 2) * pme_row(K) * elem <= 36864 && lb * 2 * K <= cap) lb *= 2;
  return lb;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct PerBufs {
  size_t o_pos, o_frc, o_ur, o_kv, o_S, o_key, o_skey, o_idx, o_sidx, o_cs, o_ce, o_tmp, o_grid, total;
};

template <typename T>
PerBufs per_layout(int N, long long nk, size_t ncell, size_t sort_bytes, size_t grid_bytes) {
  PerBufs o;
  o.o_pos = 0;
  o.o_frc = o.o_pos + al256(sizeof(T) * 16 * (size_t)N);
  o.o_ur = o.o_frc + al256(sizeof(T) * 4 * (size_t)N);
  o.o_kv = o.o_ur + al256(sizeof(T) * 3 * (size_t)N);
  o.o_S = o.o_kv + al256(sizeof(T) * 4 * (size_t)std::max(nk, 1ll));
  o.o_key = o.o_S + al256(sizeof(T) * 6 * (size_t)std::max(nk, 1ll));
  o.o_skey = o.o_key + al256(sizeof(unsigned int) * (size_t)N);
  o.o_idx = o.o_skey + al256(sizeof(unsigned int) * (size_t)N);
  o.o_sidx = o.o_idx + al256(sizeof(int) * (size_t)N);
  o.o_cs = o.o_sidx + al256(sizeof(int) * (size_t)N);
  o.o_ce = o.o_cs + al256(sizeof(int) * ncell);
  o.o_tmp = o.o_ce + al256(sizeof(int) * ncell);
  o.o_grid = o.o_tmp + al256(sort_bytes + 1);
  o.total = o.o_grid + al256(grid_bytes + 1);
  return o;
}

// Ewald sum of the cube: real space by cell list (M >= 3) or every pair (M = 0); wave
// space directly over the kept wave vectors (K = 0) or on a K^3 mesh (K > 0).
template <typename T>
gbi_status run_periodic(gbi_ctx* ctx, int N, double L, double a, double eta, const double* R, const double* Va,
                        const double* Fe, double* V, const EwaldPlan& p, int K) {
  using G = T;   // mesh precision: that of the sums
  std::vector<T> kv;
  if (K == 0) ewald_kvectors<T>(p, L, kv);
  const long long nk = (long long)kv.size() / 4;
  const int M = p.M;
  const size_t ncell = M > 0 ? (size_t)M * M * M : 1;
  size_t sort_bytes = 0;
  if (M > 0)
    GBI_CHECK(cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (const unsigned int*)nullptr, (unsigned int*)nullptr,
                                              (const int*)nullptr, (int*)nullptr, N, 0, 32, ctx->stream));
  const size_t K3 = (size_t)K * K * K;
  using C = typename Cplx<G>::t;
  using Q = typename Cplx<G>::q;
  // the mesh form keeps the K spline moduli in the wave-vector slot and the K twiddles
  // in the structure-factor slot (both sized for at least K / 4 wave vectors); its grids
  // are the staging points and the two complex grids A, B
  const long long slots = std::max(nk, (long long)K);
  const size_t mesh_bytes = K > 0 ? K3 * (sizeof(Q) + 2 * sizeof(C)) : 0;
  const PerBufs o = per_layout<T>(N, slots, ncell, sort_bytes, mesh_bytes);
  GBI_TRY(ensure(ctx, ctx->perbuf, o.total));
  char* b = static_cast<char*>(ctx->perbuf.p);
  T* pos = reinterpret_cast<T*>(b + o.o_pos);
  T* frc = reinterpret_cast<T*>(b + o.o_frc);
  T* ur = reinterpret_cast<T*>(b + o.o_ur);
  T* kvd = reinterpret_cast<T*>(b + o.o_kv);
  T* S = reinterpret_cast<T*>(b + o.o_S);
  unsigned int* key = reinterpret_cast<unsigned int*>(b + o.o_key);
  unsigned int* skey = reinterpret_cast<unsigned int*>(b + o.o_skey);
  int* idx = reinterpret_cast<int*>(b + o.o_idx);
  int* sidx = reinterpret_cast<int*>(b + o.o_sidx);
  int* cs = reinterpret_cast<int*>(b + o.o_cs);
  int* ce = reinterpret_cast<int*>(b + o.o_ce);
  if (nk > 0) {
    GBI_CHECK(cudaMemcpyAsync(kvd, kv.data(), sizeof(T) * kv.size(), cudaMemcpyHostToDevice, ctx->stream));
  }
  // records in cell order (M >= 3) or in input order (every pair)
  const int* order = nullptr;
  if (M > 0) {
    k_per_keys<<<grid1(N), 256, 0, ctx->stream>>>(N, L, M, R, key, idx);
    size_t tb = sort_bytes;
    GBI_CHECK(cub::DeviceRadixSort::SortPairs(b + o.o_tmp, tb, key, skey, idx, sidx, N, 0, 32, ctx->stream));
    GBI_CHECK(cudaMemsetAsync(cs, 0, sizeof(int) * ncell, ctx->stream));
    GBI_CHECK(cudaMemsetAsync(ce, 0, sizeof(int) * ncell, ctx->stream));
    k_per_cell_bounds<<<grid1(N), 256, 0, ctx->stream>>>(N, skey, cs, ce);
    ctx->launches += 2;
    order = sidx;
  }
  k_per_records<T><<<grid1(N), 256, 0, ctx->stream>>>(N, L, R, Fe, order, pos, frc);
  if (M > 0) {
    // slices per cell: enough blocks for a cell of mean + 4 sigma records
    const double mean = double(N) / double(ncell);
    const int slices = std::max(1, (int)std::ceil((mean + 4.0 * std::sqrt(mean) + 1.0) / kPerCellSlots));
    k_per_real_cells<T><<<dim3((unsigned)ncell, (unsigned)slices), kPerCellThreads, 0, ctx->stream>>>(
        M, L, p.rc, p.xi, pos, frc, cs, ce, ur);
  }
  else
    k_per_real_all<T><<<grid1(N, kPerThreads), kPerThreads, 0, ctx->stream>>>(N, L, p.rc, p.xi, pos, frc, ur);
  ctx->launches += 2;
  std::vector<double> bm;
  std::vector<G> bmg, twh;
  if (K == 0) {
    k_per_struct<T><<<(unsigned)((std::max(nk, 1ll) + kPerThreads - 1) / kPerThreads), kPerThreads, 0,
                      ctx->stream>>>(N, nk, kvd, pos, frc, S);
    k_per_recip<T><<<grid1(N, kPerThreads), kPerThreads, 0, ctx->stream>>>(N, nk, p.xi, a, eta, kvd, S, pos, order,
                                                                            Fe, ur, Va, V);
    ctx->launches += 2;
  } else {
    int logK = 0;
    while ((1 << logK) < K) ++logK;
    bm = pme_bmod(K);
    bmg.assign(bm.begin(), bm.end());
    // twiddles e^{-2 pi i t / K}, t < K, as (re, im) pairs
    twh.resize(2 * (size_t)K);
    for (int t = 0; t < K; ++t) {
      twh[2 * t] = G(std::cos(2.0 * kPi * t / K));
      twh[2 * t + 1] = G(-std::sin(2.0 * kPi * t / K));
    }
    G* bmd = reinterpret_cast<G*>(b + o.o_kv);
    C* twd = reinterpret_cast<C*>(b + o.o_S);
    Q* Qs = reinterpret_cast<Q*>(b + o.o_grid);
    C* A = reinterpret_cast<C*>(b + o.o_grid + K3 * sizeof(Q));
    C* B = A + K3;
    GBI_CHECK(cudaMemcpyAsync(bmd, bmg.data(), sizeof(G) * K, cudaMemcpyHostToDevice, ctx->stream));
    GBI_CHECK(cudaMemcpyAsync(twd, twh.data(), sizeof(G) * 2 * K, cudaMemcpyHostToDevice, ctx->stream));
    GBI_CHECK(cudaMemsetAsync(Qs, 0, sizeof(Q) * K3, ctx->stream));
    const unsigned lane_blocks = (unsigned)(((size_t)N * kPmeLanes + 127) / 128);
    k_pme_spread<G><<<lane_blocks, 128, 0, ctx->stream>>>(N, K, R, L, Fe, sidx, Qs);
    const int LB = pme_lines_per_block(K, sizeof(C));
    int logLB = 0;
    while ((1 << logLB) < LB) ++logLB;
    const dim3 lines((unsigned)((size_t)K * K / LB), 2);
    const size_t fsm = sizeof(C) * ((size_t)LB * pme_row(K) + K);
    // forward along z (from the staging points) and y, then x with the products and x back,
    // then y and z back
    const int logP = logLB - 2;   // 4 P rows = LB rows in shared memory
    const unsigned xblocks = (unsigned)((size_t)K * K >> logP);
    cudaError_t e = cudaSuccess;
    switch (K / 16) {
#define GBI_PME_FFT(N2)                                                                                     \
  case N2:                                                                                                  \
    k_pme_fft4<G, N2><<<lines, kPmeFftThreads, fsm, ctx->stream>>>(A, Qs, logLB, 2, 0, twd);                \
    k_pme_fft4<G, N2><<<lines, kPmeFftThreads, fsm, ctx->stream>>>(A, nullptr, logLB, 1, 0, twd);           \
    k_pme_xconv<G, N2><<<xblocks, kPmeFftThreads, fsm, ctx->stream>>>(A, B, logP, L, p.xi, bmd, twd);       \
    k_pme_fft4<G, N2><<<lines, kPmeFftThreads, fsm, ctx->stream>>>(A, nullptr, logLB, 1, 1, twd);           \
    k_pme_fft4<G, N2><<<lines, kPmeFftThreads, fsm, ctx->stream>>>(A, nullptr, logLB, 2, 1, twd);           \
    break;
      GBI_PME_FFT(1)
      GBI_PME_FFT(2)
      GBI_PME_FFT(4)
      GBI_PME_FFT(8)
      GBI_PME_FFT(16)
      GBI_PME_FFT(32)
#undef GBI_PME_FFT
      default: e = cudaErrorInvalidValue;
    }
    GBI_CHECK(e);
    k_pme_gather<G, T><<<lane_blocks, 128, 0, ctx->stream>>>(N, K, R, L, Fe, sidx, A, B, p.xi, a, eta, ur, Va, V);
    ctx->launches += 7;
  }
  GBI_CHECK(cudaGetLastError());
  // the host copies (wave vectors, B-spline moduli) must outlive the transfers
  GBI_CHECK(cudaStreamSynchronize(ctx->stream));
  return GBI_OK;
}

// the mesh of a split: the smallest power of 2 with K >= 5 xi L (at least 16)
int pme_mesh(const EwaldPlan& p, double L) {
  int K = 16;
  while (K < kPmeMeshPerXiL * p.xi * L) K <<= 1;
  return K;
}

// Estimated seconds of the two wave-space forms on this GPU (rates measured on GB300 for
// these kernels: ~7e10 erfc pair terms or wave terms per second, ~2e11 cell-list pair
// checks, mesh passes at ~5 TB/s over 240 bytes per FP32 mesh point, ~3e11 spreading
// atomics per second).
double cost_real(int N, const EwaldPlan& p) {
  if (p.M == 0) return double(N) * N / 7.0e10;
  return 27.0 * double(N) * N / (double(p.M) * p.M * p.M) / 2.0e11;
}
double cost_direct(int N, const EwaldPlan& p) { return cost_real(N, p) + 2.0 * N * double(p.nk) / 7.0e10; }
double cost_mesh(int N, const EwaldPlan& p, int K) {
  const double K3 = double(K) * K * K;
  return cost_real(N, p) + K3 * 240.0 / 5.0e12 + 3.0 * N * kPmeOrder * kPmeOrder * kPmeOrder / 3.0e11 + 5.0e-5;
}

}  // namespace
}  // namespace gbi

using namespace gbi;

extern "C" gbi_status gbi_periodic_superpose(gbi_ctx* ctx, const gbi_params* prm, int N, double L, const double* R,
                                             const double* Va, const double* Fe, double* V, int* cells_per_side,
                                             int* mesh, double* xi, long long* n_wave) {
  if (!ctx || !valid_params(prm) || N < 0 || !(L > 0)) return GBI_ERR_ARG;
  const int want_cells = cells_per_side ? *cells_per_side : 0;
  const int want_mesh = mesh ? *mesh : 0;
  if (want_mesh > 0 && (want_mesh < 16 || want_mesh > 512 || (want_mesh & (want_mesh - 1)) != 0 || want_cells < 0))
    return GBI_ERR_ARG;
  if (N == 0) return GBI_OK;
  if (!R || !Va || !Fe || !V) return GBI_ERR_ARG;
  cudaSetDevice(ctx->device);
  const bool fp32 = prm->precision == 1 || prm->precision == 3;
  EwaldPlan p = ewald_plan(N, L, fp32, want_cells);
  int K = 0;
  if (want_mesh > 0) {
    // an imposed mesh: the cells imposed (at most 128 per side), else the most cells
    // per side that the mesh resolves (K >= 5 xi L), at least 3
    int M = want_cells;
    if (M == 0) {
      M = 3;
      while (M < 128 && (long long)(M + 1) * (M + 1) * (M + 1) <= 4 * (long long)N &&
             pme_mesh(ewald_plan_for(M + 1, L, fp32), L) <= want_mesh)
        ++M;
    }
    p = ewald_plan_for(std::max(3, std::min(M, 128)), L, fp32);
    K = want_mesh;
  } else if (want_mesh == 0 && fp32 && want_cells >= 0) {
    // the mesh where it is estimated cheaper, with the cells per side that minimise it
    // (meshes up to 512^3; FP64 keeps the direct sum, whose truncation is ~1e-13)
    double best = cost_direct(N, p);
    for (int M = 3; (long long)M * M * M <= 4 * (long long)N; ++M) {
      if (want_cells > 0 && M != p.M) continue;
      const EwaldPlan q = ewald_plan_for(M, L, true);
      const int Kq = pme_mesh(q, L);
      if (Kq > 512) break;
      const double c = cost_mesh(N, q, Kq);
      if (c < best) {
        best = c;
        p = q;
        K = Kq;
      }
    }
  }
  if (cells_per_side) *cells_per_side = p.M;
  if (mesh) *mesh = K;
  if (xi) *xi = p.xi;
  if (n_wave) {
    if (K > 0) {
      *n_wave = (long long)K * K * K;
    } else {
      std::vector<float> kv;
      ewald_kvectors<float>(p, L, kv);
      *n_wave = (long long)kv.size() / 4;
    }
  }
  if (fp32) return run_periodic<float>(ctx, N, L, prm->a, prm->eta, R, Va, Fe, V, p, K);
  return run_periodic<double>(ctx, N, L, prm->a, prm->eta, R, Va, Fe, V, p, K);
}
