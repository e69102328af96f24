// Closed-form superposition pair sum for the l <= 2 mode set (Sec. IV, second form of
// Eq. mobility_matrices and Eq. propulsion_matrices; Sec. V, Eq. trap_eom).
//
// Each source sphere m carries a force F, a torque T, the one-body stresslet
// S = a Q^(20) = -(20/3) pi eta a^2 V^(20) and the one-body potential dipole
// Q^(32) = -2 pi eta a V^(32).  With rho = R_n - R_m and everything divided by 8 pi eta:
//   V_n += (1/r + 2a^2/(3r^3)) F + (1/r^3 - 2a^2/r^5)(rho.F) rho          (RPY, F^0 F^0 G)
//        + (T x rho)/r^3                                                   (rotlet)
//        - 3 (rho.S.rho) rho/r^5 + a^2 [8 (rho.S.rho) rho/r^7 - 16/5 S.rho/r^5]
//                                                   (stresslet with F^0 F^1, 4a^2/15 lap)
//        + (a^3/10) [3 (rho.d) rho/r^5 - d/r^3] * 8 pi eta                (potential dipole)
//   Omega_n += (F x rho)/r^3 + [3 (T.rho) rho/r^5 - T/r^3]/2 + 3 rho x (S.rho)/r^5
// plus the one-body terms V^a + F/(6 pi eta a) and Omega^a + T/(8 pi eta a^3).
// One warp per target sphere, lanes stride over sources staged in shared memory.
#include <type_traits>

#include "gbi_generated.cuh"
#include "gbi_internal.cuh"

namespace gbi {

namespace {


template <typename T, int WARPS, int TILE>
__global__ void __launch_bounds__(WARPS * 32) trap_kernel(const TrapArgs args) {
  constexpr bool F32 = std::is_same<T, float>::value;
  constexpr int POSW = F32 ? 6 : 3;
  __shared__ T s_pos[POSW][TILE];
  __shared__ T s_src[15][TILE];

  const int N = args.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.x * WARPS + warp;
  const bool active = n < N;
  const double inv8pe = 1.0 / (8.0 * kPi * args.eta);
  const T a = T(args.a);
  const T a2 = a * a;

  T tp[POSW];
#pragma unroll
  for (int i = 0; i < POSW; ++i) tp[i] = T(0);
  if (active) {
    if constexpr (F32) {
      const float4 h = args.pos.hi[n], lo = args.pos.lo[n];
      tp[0] = h.x; tp[1] = h.y; tp[2] = h.z; tp[3] = lo.x; tp[4] = lo.y; tp[5] = lo.z;
    } else {
      const dpos4 p = args.pos.p64[n];
      tp[0] = p.x; tp[1] = p.y; tp[2] = p.z;
    }
  }
  T v0 = 0, v1 = 0, v2 = 0, w0 = 0, w1 = 0, w2 = 0;

  for (int base = 0; base < N; base += TILE) {
    const int len = min(TILE, N - base);
    __syncthreads();
    for (int j = threadIdx.x; j < len; j += WARPS * 32) {
      const int m = base + j;
      if constexpr (F32) {
        const float4 h = args.pos.hi[m], lo = args.pos.lo[m];
        s_pos[0][j] = h.x; s_pos[1][j] = h.y; s_pos[2][j] = h.z;
        s_pos[3][j] = lo.x; s_pos[4][j] = lo.y; s_pos[5][j] = lo.z;
      } else {
        const dpos4 p = args.pos.p64[m];
        s_pos[0][j] = p.x; s_pos[1][j] = p.y; s_pos[2][j] = p.z;
      }
      const double* F = args.Fe + 3 * (size_t)m;
      const double* Tq = args.Te + 3 * (size_t)m;
      const double* vh = args.VH + 8 * (size_t)m;
      double s6[6];
      gbi_unpack2<double>(vh, s6);
      const double sf = -(5.0 / 6.0) * args.a * args.a;        // S/(8 pi eta) per V^(20)
      const double df = args.a * args.a * args.a / 10.0;        // (a^3/10) per V^(32)
      s_src[0][j] = T(F[0] * inv8pe); s_src[1][j] = T(F[1] * inv8pe); s_src[2][j] = T(F[2] * inv8pe);
      s_src[3][j] = T(Tq[0] * inv8pe); s_src[4][j] = T(Tq[1] * inv8pe); s_src[5][j] = T(Tq[2] * inv8pe);
      s_src[6][j] = T(sf * s6[0]); s_src[7][j] = T(sf * s6[1]); s_src[8][j] = T(sf * s6[2]);
      s_src[9][j] = T(sf * s6[3]); s_src[10][j] = T(sf * s6[4]); s_src[11][j] = T(sf * s6[5]);
      // V^(32) packed (y, z, x)
      s_src[12][j] = T(df * vh[7]); s_src[13][j] = T(df * vh[5]); s_src[14][j] = T(df * vh[6]);
    }
    __syncthreads();
    if (active) {
      for (int j = lane; j < len; j += 32) {
        if (base + j == n) continue;
        T x, y, z;
        if constexpr (F32) {
          x = (tp[0] - s_pos[0][j]) + (tp[3] - s_pos[3][j]);
          y = (tp[1] - s_pos[1][j]) + (tp[4] - s_pos[4][j]);
          z = (tp[2] - s_pos[2][j]) + (tp[5] - s_pos[5][j]);
        } else {
          x = tp[0] - s_pos[0][j];
          y = tp[1] - s_pos[1][j];
          z = tp[2] - s_pos[2][j];
        }
        const T r2 = x * x + y * y + z * z;
        T ri;
        if constexpr (F32) ri = rsqrtf(r2); else ri = rsqrt(r2);
        const T ri2 = ri * ri, ri3 = ri * ri2, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
        const T Fx = s_src[0][j], Fy = s_src[1][j], Fz = s_src[2][j];
        const T Tx = s_src[3][j], Ty = s_src[4][j], Tz = s_src[5][j];
        const T Sxx = s_src[6][j], Sxy = s_src[7][j], Sxz = s_src[8][j];
        const T Syy = s_src[9][j], Syz = s_src[10][j], Szz = s_src[11][j];
        const T dx = s_src[12][j], dy = s_src[13][j], dz = s_src[14][j];
        // RPY
        const T rF = x * Fx + y * Fy + z * Fz;
        const T c1 = ri + T(2.0 / 3.0) * a2 * ri3;
        const T c2 = (ri3 - T(2) * a2 * ri5) * rF;
        // stresslet
        const T Sx = Sxx * x + Sxy * y + Sxz * z;
        const T Sy = Sxy * x + Syy * y + Syz * z;
        const T Sz = Sxz * x + Syz * y + Szz * z;
        const T rSr = x * Sx + y * Sy + z * Sz;
        const T cs = (T(8) * a2 * ri7 - T(3) * ri5) * rSr;
        const T cs2 = T(-16.0 / 5.0) * a2 * ri5;
        // dipole
        const T rd = x * dx + y * dy + z * dz;
        const T cd = T(3) * ri5 * rd;
        // torque
        const T rT = x * Tx + y * Ty + z * Tz;
        const T ct = T(1.5) * ri5 * rT;
        v0 += c1 * Fx + c2 * x + (Ty * z - Tz * y) * ri3 + cs * x + cs2 * Sx + cd * x - ri3 * dx;
        v1 += c1 * Fy + c2 * y + (Tz * x - Tx * z) * ri3 + cs * y + cs2 * Sy + cd * y - ri3 * dy;
        v2 += c1 * Fz + c2 * z + (Tx * y - Ty * x) * ri3 + cs * z + cs2 * Sz + cd * z - ri3 * dz;
        const T t3 = T(3) * ri5;
        w0 += (Fy * z - Fz * y) * ri3 + ct * x - T(0.5) * ri3 * Tx + t3 * (y * Sz - z * Sy);
        w1 += (Fz * x - Fx * z) * ri3 + ct * y - T(0.5) * ri3 * Ty + t3 * (z * Sx - x * Sz);
        w2 += (Fx * y - Fy * x) * ri3 + ct * z - T(0.5) * ri3 * Tz + t3 * (x * Sy - y * Sx);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    w0 += __shfl_xor_sync(0xffffffffu, w0, o);
    w1 += __shfl_xor_sync(0xffffffffu, w1, o);
    w2 += __shfl_xor_sync(0xffffffffu, w2, o);
  }
  if (active && lane == 0) {
    const double mt = 1.0 / (6.0 * kPi * args.eta * args.a);
    const double mr = 1.0 / (8.0 * kPi * args.eta * args.a * args.a * args.a);
    const double* F = args.Fe + 3 * (size_t)n;
    const double* Tq = args.Te + 3 * (size_t)n;
    const double* va = args.Va + 3 * (size_t)n;
    const double* oa = args.Oa + 3 * (size_t)n;
    double* V = args.V + 3 * (size_t)n;
    double* O = args.Om + 3 * (size_t)n;
    V[0] = va[0] + mt * F[0] + double(v0);
    V[1] = va[1] + mt * F[1] + double(v1);
    V[2] = va[2] + mt * F[2] + double(v2);
    O[0] = oa[0] + mr * Tq[0] + double(w0);
    O[1] = oa[1] + mr * Tq[1] + double(w1);
    O[2] = oa[2] + mr * Tq[2] + double(w2);
  }
}

}  // namespace

double trap_flops() {
  // rho (9, two-float), r^2 (5), rsqrt (1), powers (4), RPY (5 + 5 + 4), stresslet S.rho (15),
  // rho.S.rho (5), coefficients (7), dipole (5 + 2), torque (5 + 2), V update (3 x 22),
  // Omega update (3 x 17)
  return 9 + 5 + 1 + 4 + 14 + 15 + 5 + 7 + 7 + 7 + 66 + 51;
}

cudaError_t launch_trap(const TrapArgs& args, int precision, cudaStream_t stream) {
  constexpr int WARPS = 8;
  if (args.N <= 0) return cudaSuccess;
  const dim3 grid((args.N + WARPS - 1) / WARPS), block(WARPS * 32);
  if (precision == 1) {
    trap_kernel<float, WARPS, 256><<<grid, block, 0, stream>>>(args);
  } else {
    trap_kernel<double, WARPS, 128><<<grid, block, 0, stream>>>(args);
  }
  return cudaGetLastError();
}

}  // namespace gbi
