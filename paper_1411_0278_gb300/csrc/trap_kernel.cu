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

// V = V^a + F/(6 pi eta a) + sum_split partial, Omega likewise (fixed split order).
template <typename T>
__global__ void trap_finish(const TrapArgs args, const T* __restrict__ partial, int nsplit) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= args.N) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int s = 0; s < nsplit; ++s) {
    const T* p = partial + ((size_t)s * args.N + n) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] += double(p[c]);
  }
  const double mt = 1.0 / (6.0 * kPi * args.eta * args.a);
  const double mr = 1.0 / (8.0 * kPi * args.eta * args.a * args.a * args.a);
  for (int c = 0; c < 3; ++c) {
    args.V[3 * (size_t)n + c] = args.Va[3 * (size_t)n + c] + mt * args.Fe[3 * (size_t)n + c] + acc[c];
    args.Om[3 * (size_t)n + c] = args.Oa[3 * (size_t)n + c] + mr * args.Te[3 * (size_t)n + c] + acc[3 + c];
  }
}

constexpr int kTI = 4, kThreads = 128;

template <typename T, int TILE>
cudaError_t trap_launch_t(const TrapArgs& args, void* scratch, int nsplit, cudaStream_t stream) {
  T* rec = reinterpret_cast<T*>(scratch);
  T* partial = rec + (size_t)args.N * kRec;
  trap_pack<T><<<(args.N + 255) / 256, 256, 0, stream>>>(args, rec);
  const int chunk = (args.N + nsplit - 1) / nsplit;
  const dim3 grid((args.N + kThreads * kTI - 1) / (kThreads * kTI), nsplit);
  trap_pairs<T, kTI, kThreads, TILE><<<grid, kThreads, 0, stream>>>(args, rec, chunk, partial);
  trap_finish<T><<<(args.N + 255) / 256, 256, 0, stream>>>(args, partial, nsplit);
  return cudaGetLastError();
}

}  // namespace

double trap_flops() {
  // rho (9, two-float), r^2 (5), rsqrt (1), powers (4), RPY coefficients (5 + 5 + 4),
  // S.rho (15), rho.S.rho (5), rho.d (5), rho.T (5), radial coefficient (8), V update (3 x 16),
  // Omega update (4 + 3 x 15)
  return 9 + 5 + 1 + 4 + 14 + 15 + 5 + 5 + 5 + 8 + 48 + 49;
}

int trap_splits(int N) {
  // about four blocks per SM on 152 SMs, at least 64 sources per split
  const int tblocks = (N + kThreads * kTI - 1) / (kThreads * kTI);
  int s = (608 + tblocks - 1) / tblocks;
  const int maxs = (N + 63) / 64;
  if (s > maxs) s = maxs;
  return s < 1 ? 1 : s;
}

size_t trap_scratch_bytes(int N, int precision) {
  const size_t w = precision == 1 ? sizeof(float) : sizeof(double);
  return w * ((size_t)N * kRec + (size_t)trap_splits(N) * N * 6) + 256;
}

// Three launches: record packing, pair sums per split, fixed-order reduction.
cudaError_t launch_trap(const TrapArgs& args, int precision, void* scratch, cudaStream_t stream) {
  if (args.N <= 0) return cudaSuccess;
  const int ns = trap_splits(args.N);
  if (precision == 1) return trap_launch_t<float, 128>(args, scratch, ns, stream);
  return trap_launch_t<double, 64>(args, scratch, ns, stream);
}

}  // namespace gbi
