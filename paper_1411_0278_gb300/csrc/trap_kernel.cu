// Closed-form superposition pair sum for the l <= 2 mode set (Sec. IV, second form of
// Eq. mobility_matrices and Eq. propulsion_matrices; Sec. V, Eq. trap_eom).
//
// Each source sphere m carries a force F, a torque T, the one-body stresslet
// S = a Q^(20) = -(20/3) pi eta a^2 V^(20) and the one-body potential dipole
// Q^(32) = -2 pi eta a V^(32).  With rho = R_n - R_m and F, T, S divided by 8 pi eta:
//   V_n += (1/r + 2a^2/(3r^3)) F + (1/r^3 - 2a^2/r^5)(rho.F) rho          (RPY, F^0 F^0 G)
//        + (T x rho)/r^3                                                   (rotlet)
//        - 3 (rho.S.rho) rho/r^5 + a^2 [8 (rho.S.rho) rho/r^7 - 16/5 S.rho/r^5]
//                                                   (stresslet with F^0 F^1, 4a^2/15 lap)
//        + (a^3/10) [3 (rho.d) rho/r^5 - d/r^3]                           (potential dipole)
//   Omega_n += (F x rho)/r^3 + [3 (T.rho) rho/r^5 - T/r^3]/2 + 3 rho x (S.rho)/r^5
// plus the one-body terms V^a + F/(6 pi eta a) and Omega^a + T/(8 pi eta a^3).
//
// Layout: a prologue kernel packs every source into one 24-word record (position
// hi/lo or FP64 position, F, T, S, d).  The pair kernel gives each thread TI target
// spheres; all threads of a block walk the same source records in shared memory
// (broadcast, vectorised reads), so each record load serves TI pairs.  Sources are
// split across blockIdx.y; every split writes its partial sums to scratch and a
// final kernel adds them in a fixed order (deterministic) together with the one-body
// terms, in FP64.
#include <type_traits>

#include "df.cuh"
#include "gbi_generated.cuh"
#include "gbi_internal.cuh"

namespace gbi {

namespace {

constexpr int kRec = 24;   // words per source record

template <typename T>
__global__ void trap_pack(const TrapArgs args, T* __restrict__ rec) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= args.N) return;
  constexpr bool F32 = std::is_same<T, float>::value;
  const double inv8pe = 1.0 / (8.0 * kPi * args.eta);
  const double* F = args.Fe + 3 * (size_t)m;
  const double* Tq = args.Te + 3 * (size_t)m;
  const double* vh = args.VH + 8 * (size_t)m;
  double s6[6];
  gbi_unpack2<double>(vh, s6);
  const double sf = -(5.0 / 6.0) * args.a * args.a;        // S/(8 pi eta) per V^(20)
  const double df = args.a * args.a * args.a / 10.0;        // (a^3/10) per V^(32)
  T* r = rec + (size_t)m * kRec;
  if constexpr (F32) {
    const float4 h = args.pos.hi[m], lo = args.pos.lo[m];
    r[0] = h.x; r[1] = h.y; r[2] = h.z; r[3] = lo.x; r[4] = lo.y; r[5] = lo.z;
  } else {
    const dpos4 p = args.pos.p64[m];
    r[0] = p.x; r[1] = p.y; r[2] = p.z; r[3] = 0; r[4] = 0; r[5] = 0;
  }
  r[6] = T(F[0] * inv8pe); r[7] = T(F[1] * inv8pe); r[8] = T(F[2] * inv8pe);
  r[9] = T(Tq[0] * inv8pe); r[10] = T(Tq[1] * inv8pe); r[11] = T(Tq[2] * inv8pe);
  for (int i = 0; i < 6; ++i) r[12 + i] = T(sf * s6[i]);
  // V^(32) packed (y, z, x)
  r[18] = T(df * vh[7]); r[19] = T(df * vh[5]); r[20] = T(df * vh[6]);
  // -T/2 (divided by 8 pi eta) for the rotlet-dipole term of Omega
  r[21] = T(-0.5 * Tq[0] * inv8pe); r[22] = T(-0.5 * Tq[1] * inv8pe); r[23] = T(-0.5 * Tq[2] * inv8pe);
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = dpos4; };

template <typename T>
__device__ __forceinline__ T trap_rsqrt(T v) {
  if constexpr (std::is_same<T, float>::value) return rsqrtf(v);
  else return rsqrt(v);
}

// The pair terms of source j of the tile (sphere m) for the thread's TI targets n0 + t.
// SELF: the tile may hold one of those targets, which is then skipped.  Each sum is an
// FMA chain: the rotlet and potential dipole share ri3 (T x rho - d), the torque's own
// rotlet-dipole term rides on the force rotlet (F x rho - T/2, with -T/2 in the record).
template <typename T, int TI, bool SELF>
__device__ __forceinline__ void trap_source(const T* __restrict__ s_rec, int j, int m, int n0, const T* px,
                                            const T* py, const T* pz, const T* lx, const T* ly, const T* lz, T a2,
                                            T* v0, T* v1, T* v2, T* w0, T* w1, T* w2) {
  constexpr bool F32 = std::is_same<T, float>::value;
  using V4 = typename Vec4<T>::type;
  const V4* r4 = reinterpret_cast<const V4*>(s_rec + j * kRec);
  const V4 q0 = r4[0], q1 = r4[1], q2 = r4[2], q3 = r4[3], q4 = r4[4], q5 = r4[5];
  const T sx = q0.x, sy = q0.y, sz = q0.z, slx = q0.w, sly = q1.x, slz = q1.y;
  const T Fx = q1.z, Fy = q1.w, Fz = q2.x;
  const T Tx = q2.y, Ty = q2.z, Tz = q2.w;
  const T Sxx = q3.x, Sxy = q3.y, Sxz = q3.z, Syy = q3.w, Syz = q4.x, Szz = q4.y;
  const T dx = q4.z, dy = q4.w, dz = q5.x;
  const T hx = q5.y, hy = q5.z, hz = q5.w;   // -T/2
  const T c23 = T(2.0 / 3.0) * a2, c2a = T(-2) * a2, c8a = T(8) * a2, c165 = T(-16.0 / 5.0) * a2;
#pragma unroll
  for (int t = 0; t < TI; ++t) {
    if (SELF && m == n0 + t) continue;
    T x, y, z;
    if constexpr (F32) {
      x = (px[t] - sx) + (lx[t] - slx);
      y = (py[t] - sy) + (ly[t] - sly);
      z = (pz[t] - sz) + (lz[t] - slz);
    } else {
      x = px[t] - sx;
      y = py[t] - sy;
      z = pz[t] - sz;
    }
    const T r2 = gbi_fmac(z, z, gbi_fmac(y, y, x * x));
    const T ri = trap_rsqrt(r2);
    const T ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
    const T rF = gbi_fmac(z, Fz, gbi_fmac(y, Fy, x * Fx));
    const T Sx = gbi_fmac(Sxz, z, gbi_fmac(Sxy, y, Sxx * x));
    const T Sy = gbi_fmac(Syz, z, gbi_fmac(Syy, y, Sxy * x));
    const T Sz = gbi_fmac(Szz, z, gbi_fmac(Syz, y, Sxz * x));
    const T rSr = gbi_fmac(z, Sz, gbi_fmac(y, Sy, x * Sx));
    const T rd = gbi_fmac(z, dz, gbi_fmac(y, dy, x * dx));
    const T rT = gbi_fmac(z, Tz, gbi_fmac(y, Ty, x * Tx));
    const T c1 = gbi_fmac(c23, ri3, ri);
    const T t3 = T(3) * ri5;
    // common radial coefficient of rho in V: RPY + stresslet + dipole
    const T cx = gbi_fmac(gbi_fmac(c2a, ri5, ri3), rF, gbi_fmac(gbi_fmac(c8a, ri7, -t3), rSr, t3 * rd));
    const T cs2 = c165 * ri5;
    // (T x rho - d) and (F x rho - T/2)
    const T u0 = gbi_fmac(Ty, z, gbi_fmac(-Tz, y, -dx));
    const T u1 = gbi_fmac(Tz, x, gbi_fmac(-Tx, z, -dy));
    const T u2 = gbi_fmac(Tx, y, gbi_fmac(-Ty, x, -dz));
    v0[t] = gbi_fmac(ri3, u0, gbi_fmac(cs2, Sx, gbi_fmac(cx, x, gbi_fmac(c1, Fx, v0[t]))));
    v1[t] = gbi_fmac(ri3, u1, gbi_fmac(cs2, Sy, gbi_fmac(cx, y, gbi_fmac(c1, Fy, v1[t]))));
    v2[t] = gbi_fmac(ri3, u2, gbi_fmac(cs2, Sz, gbi_fmac(cx, z, gbi_fmac(c1, Fz, v2[t]))));
    const T e0 = gbi_fmac(Fy, z, gbi_fmac(-Fz, y, hx));
    const T e1 = gbi_fmac(Fz, x, gbi_fmac(-Fx, z, hy));
    const T e2 = gbi_fmac(Fx, y, gbi_fmac(-Fy, x, hz));
    const T ct = (T(1.5) * ri5) * rT;
    const T tx = t3 * x, ty = t3 * y, tz = t3 * z;
    w0[t] = gbi_fmac(ty, Sz, gbi_fmac(-tz, Sy, gbi_fmac(ct, x, gbi_fmac(ri3, e0, w0[t]))));
    w1[t] = gbi_fmac(tz, Sx, gbi_fmac(-tx, Sz, gbi_fmac(ct, y, gbi_fmac(ri3, e1, w1[t]))));
    w2[t] = gbi_fmac(tx, Sy, gbi_fmac(-ty, Sx, gbi_fmac(ct, z, gbi_fmac(ri3, e2, w2[t]))));
  }
}

// Two FP32 values per instruction (the paired FFMA2 / FMUL2 / FADD2 of sm_100 and later).
// Each element is rounded exactly as the scalar operation rounds it, so the paired pass
// gives the scalar pass's results bit for bit; it halves the issued FP32 instructions,
// not the FMA pipe's work (a paired FMA occupies the pipe for two lanes' worth).
struct f2 {
  float2 v;
  __device__ __forceinline__ f2() {}
  __device__ __forceinline__ explicit f2(float s) : v(make_float2(s, s)) {}
  __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
  __device__ __forceinline__ explicit f2(float2 p) : v(p) {}
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(-a.v.x, -a.v.y); }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return a + (-b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f2 rsqrt2(f2 a) { return f2(rsqrtf(a.v.x), rsqrtf(a.v.y)); }

// trap_source for FP32 targets taken two at a time: pair g holds targets n0 + 2g (x) and
// n0 + 2g + 1 (y).  The source record sits in shared memory with every word duplicated
// ((w, w) pairs), so each 16-byte load yields two broadcast operands.  The operations and
// their order per element are those of trap_source.  SELF: the tile may hold one of the
// thread's targets.  Its rho is exactly zero (same position words), so with 1/r set to 0
// for that lane every one of its terms is a product with 0 and its sums do not change.
template <int TG, bool SELF>
__device__ __forceinline__ void trap_source_f2(const float4* __restrict__ s_dup, int j, int m, int n0, const f2* px, const f2* py,
                                               const f2* pz, const f2* lx, const f2* ly, const f2* lz, f2 a2,
                                               f2* v0, f2* v1, f2* v2, f2* w0, f2* w1, f2* w2) {
  const float4* r4 = s_dup + j * (kRec / 2);
  f2 q[kRec];
#pragma unroll
  for (int i = 0; i < kRec / 2; ++i) {
    const float4 w = r4[i];
    q[2 * i] = f2(w.x, w.y);
    q[2 * i + 1] = f2(w.z, w.w);
  }
  const f2 sx = q[0], sy = q[1], sz = q[2], slx = q[3], sly = q[4], slz = q[5];
  const f2 Fx = q[6], Fy = q[7], Fz = q[8];
  const f2 Tx = q[9], Ty = q[10], Tz = q[11];
  const f2 Sxx = q[12], Sxy = q[13], Sxz = q[14], Syy = q[15], Syz = q[16], Szz = q[17];
  const f2 dx = q[18], dy = q[19], dz = q[20];
  const f2 hx = q[21], hy = q[22], hz = q[23];
  const f2 c23 = f2(2.0f / 3.0f) * a2, c2a = f2(-2.0f) * a2, c8a = f2(8.0f) * a2, c165 = f2(-16.0f / 5.0f) * a2;
#pragma unroll
  for (int g = 0; g < TG; ++g) {
    const f2 x = (px[g] - sx) + (lx[g] - slx);
    const f2 y = (py[g] - sy) + (ly[g] - sly);
    const f2 z = (pz[g] - sz) + (lz[g] - slz);
    const f2 r2 = fma2(z, z, fma2(y, y, x * x));
    f2 ri = rsqrt2(r2);
    if (SELF) {
      if (m == n0 + 2 * g) ri.v.x = 0.0f;
      if (m == n0 + 2 * g + 1) ri.v.y = 0.0f;
    }
    const f2 ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
    const f2 rF = fma2(z, Fz, fma2(y, Fy, x * Fx));
    const f2 Sx = fma2(Sxz, z, fma2(Sxy, y, Sxx * x));
    const f2 Sy = fma2(Syz, z, fma2(Syy, y, Sxy * x));
    const f2 Sz = fma2(Szz, z, fma2(Syz, y, Sxz * x));
    const f2 rSr = fma2(z, Sz, fma2(y, Sy, x * Sx));
    const f2 rd = fma2(z, dz, fma2(y, dy, x * dx));
    const f2 rT = fma2(z, Tz, fma2(y, Ty, x * Tx));
    const f2 c1 = fma2(c23, ri3, ri);
    const f2 t3 = f2(3.0f) * ri5;
    const f2 cx = fma2(fma2(c2a, ri5, ri3), rF, fma2(fma2(c8a, ri7, -t3), rSr, t3 * rd));
    const f2 cs2 = c165 * ri5;
    const f2 u0 = fma2(Ty, z, fma2(-Tz, y, -dx));
    const f2 u1 = fma2(Tz, x, fma2(-Tx, z, -dy));
    const f2 u2 = fma2(Tx, y, fma2(-Ty, x, -dz));
    v0[g] = fma2(ri3, u0, fma2(cs2, Sx, fma2(cx, x, fma2(c1, Fx, v0[g]))));
    v1[g] = fma2(ri3, u1, fma2(cs2, Sy, fma2(cx, y, fma2(c1, Fy, v1[g]))));
    v2[g] = fma2(ri3, u2, fma2(cs2, Sz, fma2(cx, z, fma2(c1, Fz, v2[g]))));
    const f2 e0 = fma2(Fy, z, fma2(-Fz, y, hx));
    const f2 e1 = fma2(Fz, x, fma2(-Fx, z, hy));
    const f2 e2 = fma2(Fx, y, fma2(-Fy, x, hz));
    const f2 ct = (f2(1.5f) * ri5) * rT;
    const f2 tx = t3 * x, ty = t3 * y, tz = t3 * z;
    w0[g] = fma2(ty, Sz, fma2(-tz, Sy, fma2(ct, x, fma2(ri3, e0, w0[g]))));
    w1[g] = fma2(tz, Sx, fma2(-tx, Sz, fma2(ct, y, fma2(ri3, e1, w1[g]))));
    w2[g] = fma2(tx, Sy, fma2(-ty, Sx, fma2(ct, z, fma2(ri3, e2, w2[g]))));
  }
}

// FP32 pair pass with paired instructions: as trap_pairs, TI = 2 TG targets per thread.
constexpr int kMinBlocks32 = 4;   // resident blocks per SM the FP32 pass is compiled for
template <int TG, int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS, kMinBlocks32) trap_pairs_f2(const TrapArgs args, const float* __restrict__ rec, int chunk,
                                                         float* __restrict__ partial) {
  constexpr int TI = 2 * TG;
  __shared__ __align__(16) float4 s_dup[TILE * kRec / 2];
  const int N = args.N;
  const int n0 = (blockIdx.x * THREADS + threadIdx.x) * TI;
  const int m_begin = blockIdx.y * chunk;
  const int m_end = min(N, m_begin + chunk);
  const f2 a2(float(args.a * args.a));
  const int blk_n0 = blockIdx.x * THREADS * TI, blk_n1 = blk_n0 + THREADS * TI;

  f2 px[TG], py[TG], pz[TG], lx[TG], ly[TG], lz[TG];
  f2 v0[TG], v1[TG], v2[TG], w0[TG], w1[TG], w2[TG];
#pragma unroll
  for (int g = 0; g < TG; ++g) {
    const int na = min(n0 + 2 * g, N - 1), nb = min(n0 + 2 * g + 1, N - 1);
    const float4 ha = args.pos.hi[na], la = args.pos.lo[na], hb = args.pos.hi[nb], lb = args.pos.lo[nb];
    px[g] = f2(ha.x, hb.x); py[g] = f2(ha.y, hb.y); pz[g] = f2(ha.z, hb.z);
    lx[g] = f2(la.x, lb.x); ly[g] = f2(la.y, lb.y); lz[g] = f2(la.z, lb.z);
    v0[g] = v1[g] = v2[g] = w0[g] = w1[g] = w2[g] = f2(0.0f);
  }

  for (int base = m_begin; base < m_end; base += TILE) {
    const int len = min(TILE, m_end - base);
    __syncthreads();
    {
      const float2* src = reinterpret_cast<const float2*>(rec + (size_t)base * kRec);
      for (int i = threadIdx.x; i < len * (kRec / 2); i += THREADS) {
        const float2 w = src[i];
        s_dup[i] = make_float4(w.x, w.x, w.y, w.y);
      }
    }
    __syncthreads();
    // only a tile that holds one of this block's targets can hold a thread's own sphere
    const bool self_tile = base < blk_n1 && base + len > blk_n0;
    if (self_tile) {
      for (int j = 0; j < len; ++j)
        trap_source_f2<TG, true>(s_dup, j, base + j, n0, px, py, pz, lx, ly, lz, a2, v0, v1, v2, w0, w1, w2);
    } else {
      for (int j = 0; j < len; ++j)
        trap_source_f2<TG, false>(s_dup, j, base + j, n0, px, py, pz, lx, ly, lz, a2, v0, v1, v2, w0, w1, w2);
    }
  }
#pragma unroll
  for (int t = 0; t < TI; ++t) {
    const int n = n0 + t;
    if (n < N) {
      const int g = t >> 1;
      const bool hi = t & 1;
      float* o = partial + ((size_t)blockIdx.y * N + n) * 6;
      o[0] = hi ? v0[g].v.y : v0[g].v.x; o[1] = hi ? v1[g].v.y : v1[g].v.x; o[2] = hi ? v2[g].v.y : v2[g].v.x;
      o[3] = hi ? w0[g].v.y : w0[g].v.x; o[4] = hi ? w1[g].v.y : w1[g].v.x; o[5] = hi ? w2[g].v.y : w2[g].v.x;
    }
  }
}

// partial[split][n][6] = sum over this split's sources of the pair terms for target n
template <typename T, int TI, int THREADS, int TILE>
__global__ void __launch_bounds__(THREADS) trap_pairs(const TrapArgs args, const T* __restrict__ rec,
                                                      int chunk, T* __restrict__ partial) {
  constexpr bool F32 = std::is_same<T, float>::value;
  using V4 = typename Vec4<T>::type;
  __shared__ __align__(32) T s_rec[TILE * kRec];
  const int N = args.N;
  const int n0 = (blockIdx.x * THREADS + threadIdx.x) * TI;
  const int m_begin = blockIdx.y * chunk;
  const int m_end = min(N, m_begin + chunk);
  const T a2 = T(args.a * args.a);
  const int blk_n0 = blockIdx.x * THREADS * TI, blk_n1 = blk_n0 + THREADS * TI;

  T px[TI], py[TI], pz[TI], lx[TI], ly[TI], lz[TI];
  T v0[TI], v1[TI], v2[TI], w0[TI], w1[TI], w2[TI];
#pragma unroll
  for (int t = 0; t < TI; ++t) {
    const int n = min(n0 + t, N - 1);
    if constexpr (F32) {
      const float4 h = args.pos.hi[n], lo = args.pos.lo[n];
      px[t] = h.x; py[t] = h.y; pz[t] = h.z; lx[t] = lo.x; ly[t] = lo.y; lz[t] = lo.z;
    } else {
      const dpos4 p = args.pos.p64[n];
      px[t] = p.x; py[t] = p.y; pz[t] = p.z; lx[t] = 0; ly[t] = 0; lz[t] = 0;
    }
    v0[t] = v1[t] = v2[t] = w0[t] = w1[t] = w2[t] = T(0);
  }

  for (int base = m_begin; base < m_end; base += TILE) {
    const int len = min(TILE, m_end - base);
    __syncthreads();
    {
      const V4* src = reinterpret_cast<const V4*>(rec + (size_t)base * kRec);
      V4* dst = reinterpret_cast<V4*>(s_rec);
      for (int i = threadIdx.x; i < len * (kRec / 4); i += THREADS) dst[i] = src[i];
    }
    __syncthreads();
    // only a tile that holds one of this block's targets can hold a thread's own sphere
    const bool self_tile = base < blk_n1 && base + len > blk_n0;
    if (self_tile) {
      for (int j = 0; j < len; ++j) trap_source<T, TI, true>(s_rec, j, base + j, n0, px, py, pz, lx, ly, lz, a2, v0, v1, v2,
                                                            w0, w1, w2);
    } else {
      for (int j = 0; j < len; ++j) trap_source<T, TI, false>(s_rec, j, base + j, n0, px, py, pz, lx, ly, lz, a2, v0, v1, v2,
                                                             w0, w1, w2);
    }
  }
#pragma unroll
  for (int t = 0; t < TI; ++t) {
    const int n = n0 + t;
    if (n < N) {
      T* o = partial + ((size_t)blockIdx.y * N + n) * 6;
      o[0] = v0[t]; o[1] = v1[t]; o[2] = v2[t]; o[3] = w0[t]; o[4] = w1[t]; o[5] = w2[t];
    }
  }
}

// V = V^a + F/(6 pi eta a) + sum_split partial, Omega likewise (fixed split order).  One
// thread per (sphere, component), component fastest, so the split rows are read coalesced;
// eight splits' loads are issued before their (ordered) FP64 additions.  mt = 1/(6 pi eta a),
// mr = 1/(8 pi eta a^3).
template <typename T>
__global__ void trap_finish(const TrapArgs args, const T* __restrict__ partial, int nsplit, double mt, double mr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long rows = 6LL * args.N;
  if (i >= rows) return;
  const long long n = i / 6;
  const int c = (int)(i - 6 * n);
  double acc = 0.0;
  int s = 0;
  for (; s + 8 <= nsplit; s += 8) {
    T p[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) p[u] = partial[(long long)(s + u) * rows + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += double(p[u]);
  }
  if (s < nsplit) {
    T p[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) p[u] = s + u < nsplit ? partial[(long long)(s + u) * rows + i] : T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (s + u < nsplit) acc += double(p[u]);
  }
  if (c < 3)
    args.V[3 * n + c] = args.Va[3 * n + c] + mt * args.Fe[3 * n + c] + acc;
  else
    args.Om[3 * n + c - 3] = args.Oa[3 * n + c - 3] + mr * args.Te[3 * n + c - 3] + acc;
}

// targets per thread: FP32 in kTG32 pairs, FP64 kTI64 one at a time
constexpr int kTG32 = 2, kTI64 = 4, kThreads = 128;
constexpr int trap_ti(int precision) { return precision == 1 ? 2 * kTG32 : kTI64; }

template <typename T, int TILE>
cudaError_t trap_launch_t(const TrapArgs& args, void* scratch, int nsplit, cudaStream_t stream) {
  T* rec = reinterpret_cast<T*>(scratch);
  T* partial = rec + (size_t)args.N * kRec;
  trap_pack<T><<<(args.N + 255) / 256, 256, 0, stream>>>(args, rec);
  const int chunk = (args.N + nsplit - 1) / nsplit;
  constexpr int TI = trap_ti(std::is_same<T, float>::value ? 1 : 0);
  const dim3 grid((args.N + kThreads * TI - 1) / (kThreads * TI), nsplit);
  if constexpr (std::is_same<T, float>::value)
    trap_pairs_f2<kTG32, kThreads, TILE><<<grid, kThreads, 0, stream>>>(args, rec, chunk, partial);
  else
    trap_pairs<T, kTI64, kThreads, TILE><<<grid, kThreads, 0, stream>>>(args, rec, chunk, partial);
  const double mt = 1.0 / (6.0 * kPi * args.eta * args.a);
  const double mr = 1.0 / (8.0 * kPi * args.eta * args.a * args.a * args.a);
  trap_finish<T><<<(int)((6LL * args.N + 255) / 256), 256, 0, stream>>>(args, partial, nsplit, mt, mr);
  return cudaGetLastError();
}

}  // namespace

double trap_flops() {
  // rho (9, two-float), r^2 (5), rsqrt (1), powers (4), RPY coefficients (5 + 5 + 4),
  // S.rho (15), rho.S.rho (5), rho.d (5), rho.T (5), radial coefficient (8), V update (3 x 16),
  // Omega update (4 + 3 x 15)
  return 9 + 5 + 1 + 4 + 14 + 15 + 5 + 5 + 5 + 8 + 48 + 49;
}

// Blocks of the pair kernel resident at once on the current device (SMs x blocks per SM at
// its registers and shared memory), per precision.  Taken once per process (thread-safe
// static initialisation); every GPU this library targets has the same count.
static int trap_resident_now(int precision) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (precision == 1)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, trap_pairs_f2<kTG32, kThreads, 128>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, trap_pairs<double, kTI64, kThreads, 64>, kThreads, 0);
  return sms * per > 0 ? sms * per : 608;
}

static int trap_resident(int precision) {
  if (precision == 1) {
    static const int r32 = trap_resident_now(1);
    return r32;
  }
  static const int r64 = trap_resident_now(0);
  return r64;
}

int trap_splits(int N, int precision) {
  // as many source splits as keep every target block's splits within one wave of the
  // resident blocks (a wave and a few stragglers costs a second wave), at least 64
  // sources per split
  const int ti = trap_ti(precision);
  const int tblocks = (N + kThreads * ti - 1) / (kThreads * ti);
  int s = trap_resident(precision) / tblocks;
  const int maxs = (N + 63) / 64;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

size_t trap_scratch_bytes(int N, int precision) {
  const size_t w = precision == 1 ? sizeof(float) : sizeof(double);
  return w * ((size_t)N * kRec + (size_t)trap_splits(N, precision) * N * 6) + 256;
}

// Three launches: record packing, pair sums per split, fixed-order reduction.
cudaError_t launch_trap(const TrapArgs& args, int precision, void* scratch, cudaStream_t stream) {
  if (args.N <= 0) return cudaSuccess;
  const int ns = trap_splits(args.N, precision);
  if (precision == 1) return trap_launch_t<float, 128>(args, scratch, ns, stream);
  return trap_launch_t<double, 64>(args, scratch, ns, stream);
}

}  // namespace gbi
