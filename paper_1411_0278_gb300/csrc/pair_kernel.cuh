// Generic single-layer Galerkin pair operator (Sec. III, Eq. single_layer_yl_matrix_element).
//
// For each target sphere n (one warp) and each source sphere m != n (one lane at a
// time, sources staged in shared memory tiles) the block G_nm is applied in the
// pair frame where R_n - R_m lies along +z:
//
//   y_n += Q^T C(r) Q x_m,     Q = D(R_y(-theta)) D(R_z(-phi)),
//
// with C(r)_pq = (1/a) (a/r)^(l_p + l_q + 1) [alpha_pq + beta_pq (a/r)^2] from the
// generated tables (the F^l finite-size operators give the beta term) and D the
// rotation matrices of the packed STF basis.  All of the pair arithmetic runs in T
// (float or double); inputs and outputs are FP64.  The FP32 path forms
// rho = (hi_n - hi_m) + (lo_n - lo_m) from a two-float split of the centres, so
// rho keeps FP32 relative accuracy even far from the origin.
#pragma once

#include <type_traits>

#include "df.cuh"
#include "gbi_generated.cuh"
#include "gbi_internal.cuh"

namespace gbi {

template <int TR> struct Tab;
#define GBI_TAB(TRN)                                                                   \
  template <> struct Tab<TRN> {                                                        \
    static constexpr int D = GbiTrunc##TRN::D;                                         \
    static constexpr int NMODE = GbiTrunc##TRN::NMODE;                                 \
    static constexpr int MAXK = GbiTrunc##TRN::MAXK;                                   \
    __host__ __device__ static constexpr int k(int m) { return gbi_t##TRN##_k(m); }    \
    __host__ __device__ static constexpr int L(int m) { return gbi_t##TRN##_L(m); }    \
    __host__ __device__ static constexpr int off(int m) { return gbi_t##TRN##_off(m); } \
  };
GBI_TAB(2)
GBI_TAB(3)
GBI_TAB(4)
GBI_TAB(5)
GBI_TAB(40)
#undef GBI_TAB

template <int TR, int ROWS, int COLS, typename T>
__host__ __device__ __forceinline__ void couple(T e2, const T* xs, T* y) {
#define GBI_C(TRN, RN, CN, RV, CV)                                 \
  if constexpr (TR == TRN && ROWS == RV && COLS == CV) {           \
    gbi_t##TRN##_couple_##RN##_##CN<T>(e2, xs, y);                 \
  }
#define GBI_C3(TRN)                                                                         \
  GBI_C(TRN, all, all, 0, 0) GBI_C(TRN, all, L, 0, 1) GBI_C(TRN, all, H, 0, 2)             \
  GBI_C(TRN, L, all, 1, 0) GBI_C(TRN, L, L, 1, 1) GBI_C(TRN, L, H, 1, 2)                   \
  GBI_C(TRN, H, all, 2, 0) GBI_C(TRN, H, L, 2, 1) GBI_C(TRN, H, H, 2, 2)
  GBI_C3(2)
  GBI_C3(3)
  GBI_C3(4)
  GBI_C3(5)
  GBI_C3(40)
  GBI_C(2, P, all, 3, 0)
  GBI_C(3, P, all, 3, 0)
  GBI_C(4, P, all, 3, 0)
  GBI_C(5, P, all, 3, 0)
  GBI_C(40, P, all, 3, 0)
#undef GBI_C3
#undef GBI_C
}

template <typename T> struct DMats {
  T d1[gbi_dm1_n];
  T d2[gbi_dm2_n];
  T d3[gbi_dm3_n];
  T d4[gbi_dm4_n];
  T d5[gbi_dm5_n];   // l <= 5 only (6t); unused members cost nothing once inlined
};

template <int K, typename T>
__host__ __device__ __forceinline__ void dapply(const DMats<T>& dm, const T* in, T* out) {
  if constexpr (K == 1) gbi_dapply1<T>(dm.d1, in, out);
  if constexpr (K == 2) gbi_dapply2<T>(dm.d2, in, out);
  if constexpr (K == 3) gbi_dapply3<T>(dm.d3, in, out);
  if constexpr (K == 4) gbi_dapply4<T>(dm.d4, in, out);
  if constexpr (K == 5) gbi_dapply5<T>(dm.d5, in, out);
}
template <int K, typename T>
__host__ __device__ __forceinline__ void dapplyT(const DMats<T>& dm, const T* in, T* out) {
  if constexpr (K == 1) gbi_dapplyT1<T>(dm.d1, in, out);
  if constexpr (K == 2) gbi_dapplyT2<T>(dm.d2, in, out);
  if constexpr (K == 3) gbi_dapplyT3<T>(dm.d3, in, out);
  if constexpr (K == 4) gbi_dapplyT4<T>(dm.d4, in, out);
  if constexpr (K == 5) gbi_dapplyT5<T>(dm.d5, in, out);
}

// v scaled by (a/r)^j = ep[j]; j = 0 leaves v untouched (no multiply by one).
template <int J, typename T>
__host__ __device__ __forceinline__ T eps_pow(const T* ep, T v) {
  if constexpr (J == 0) return v;
  else return ep[J] * v;
}

// Rotate the column modes [M, MEND) of x (absolute component index) into the pair
// frame and scale by (a/r)^l: xs = (a/r)^l D_y Z x.  The scaling rides on the z
// rotation: its cos/sin factors are taken times (a/r)^l (products shared by every mode
// with the same l), so no separate multiply per component is needed.
template <int TR, typename T, int M, int MEND>
__host__ __device__ __forceinline__ void to_pair_frame(const T* x, T* xs, const T* cm, const T* sm,
                                              const DMats<T>& dm, const T* ep) {
  if constexpr (M < MEND) {
    constexpr int k = Tab<TR>::k(M);
    constexpr int o = Tab<TR>::off(M);
    constexpr int l = Tab<TR>::L(M) - 1;
    T t[2 * k + 1];
    t[k] = eps_pow<l>(ep, x[o + k]);
#pragma unroll
    for (int mm = 1; mm <= k; ++mm) {
      const T c = eps_pow<l>(ep, cm[mm]), s = eps_pow<l>(ep, sm[mm]);
      const T xp = x[o + k + mm], xn = x[o + k - mm];
      t[k + mm] = gbi_fmac(c, xp, s * xn);
      t[k - mm] = gbi_fmac(c, xn, -(s * xp));
    }
    dapply<k, T>(dm, t, xs + o);
    to_pair_frame<TR, T, M + 1, MEND>(x, xs, cm, sm, dm, ep);
  }
}

// Rotate the row modes [M, MEND) of the pair-frame result back and accumulate:
// acc += Z^T D_y^T (a/r)^(l+1) yy.  acc is indexed from the first row component R0.
// As above, (a/r)^(l+1) multiplies the z rotation's cos/sin instead of yy.
template <int TR, typename T, int M, int MEND, int R0>
__host__ __device__ __forceinline__ void from_pair_frame(const T* yy, T* acc, const T* cm, const T* sm,
                                                const DMats<T>& dm, const T* ep) {
  if constexpr (M < MEND) {
    constexpr int k = Tab<TR>::k(M);
    constexpr int o = Tab<TR>::off(M);
    constexpr int l = Tab<TR>::L(M) - 1;
    T t[2 * k + 1];
    dapplyT<k, T>(dm, yy + o, t);
    acc[o - R0 + k] = gbi_fmac(ep[l + 1], t[k], acc[o - R0 + k]);
#pragma unroll
    for (int mm = 1; mm <= k; ++mm) {
      const T c = ep[l + 1] * cm[mm], s = ep[l + 1] * sm[mm];
      const T tp = t[k + mm], tn = t[k - mm];
      acc[o - R0 + k + mm] = gbi_fmac(c, tp, gbi_fmac(-s, tn, acc[o - R0 + k + mm]));
      acc[o - R0 + k - mm] = gbi_fmac(s, tp, gbi_fmac(c, tn, acc[o - R0 + k - mm]));
    }
    from_pair_frame<TR, T, M + 1, MEND, R0>(yy, acc, cm, sm, dm, ep);
  }
}

__host__ __device__ __forceinline__ float gbi_rsqrt(float v) {
#ifdef __CUDA_ARCH__
  return rsqrtf(v);
#else
  return 1.0f / sqrtf(v);
#endif
}
__host__ __device__ __forceinline__ double gbi_rsqrt(double v) {
#ifdef __CUDA_ARCH__
  return rsqrt(v);
#else
  return 1.0 / sqrt(v);
#endif
}

__host__ __device__ __forceinline__ df gbi_rsqrt(df v) { return df_rsqrt(v); }

__device__ __forceinline__ float gbi_shfl(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double gbi_shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df gbi_shfl(df v, int o) { return df_shfl_xor(v, o); }
__host__ __device__ __forceinline__ double gbi_to_double(float v) { return double(v); }
__host__ __device__ __forceinline__ double gbi_to_double(double v) { return v; }
__host__ __device__ __forceinline__ double gbi_to_double(df v) { return df_to_double(v); }

// Row/column component and mode ranges of a pair pass.
template <int TR, int ROWS, int COLS> struct PassShape {
  static constexpr int D = Tab<TR>::D;
  static constexpr int R0 = ROWS == SET_H ? 6 : 0;
  static constexpr int R1 = ROWS == SET_P ? 3 : (ROWS == SET_L ? 6 : D);
  static constexpr int C0 = COLS == SET_H ? 6 : 0;
  static constexpr int C1 = COLS == SET_L ? 6 : D;
  static constexpr int NR = R1 - R0;
  static constexpr int NC = C1 - C0;
  static constexpr int MR0 = ROWS == SET_H ? 2 : 0;
  static constexpr int MR1 = ROWS == SET_P ? 1 : (ROWS == SET_L ? 2 : Tab<TR>::NMODE);
  static constexpr int MC0 = COLS == SET_H ? 2 : 0;
  static constexpr int MC1 = COLS == SET_L ? 2 : Tab<TR>::NMODE;
  static constexpr int MAXK_R = (ROWS == SET_L || ROWS == SET_P) ? 1 : Tab<TR>::MAXK;
  static constexpr int MAXK_C = COLS == SET_L ? 1 : Tab<TR>::MAXK;
  static constexpr int MAXK = MAXK_R > MAXK_C ? MAXK_R : MAXK_C;
};

// One ordered pair: acc[p - R0] += sum_q C-rotated block [p][q] * xl[q] for
// rho = (dx, dy, dz) = R_n - R_m, xl indexed by absolute component (columns only).
// The 1/a factor of the block is applied by the caller.
template <int TR, int ROWS, int COLS, typename T>
__host__ __device__ __forceinline__ void pair_body(T dx, T dy, T dz, T a, const T* xl, T* acc) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int MAXK = S::MAXK;
  const T rxy2 = dx * dx + dy * dy;
  const T r2 = rxy2 + dz * dz;
  const T rinv = gbi_rsqrt(r2);
  const T eps = a * rinv;
  const T e2 = eps * eps;
  // direction: theta from +z, phi in the xy plane
  const T ct = dz * rinv;
  T cphi = T(1), sphi = T(0), st = T(0);
  if (rxy2 > T(0)) {
    const T rxyinv = gbi_rsqrt(rxy2);
    cphi = dx * rxyinv;
    sphi = dy * rxyinv;
    st = rxy2 * rxyinv * rinv;
  }
  T cm[MAXK + 1], sm[MAXK + 1];
  cm[0] = T(1); sm[0] = T(0);
  cm[1] = cphi; sm[1] = sphi;
#pragma unroll
  for (int mm = 2; mm <= MAXK; ++mm) {
    cm[mm] = gbi_fmac(cm[mm - 1], cphi, -(sm[mm - 1] * sphi));
    sm[mm] = gbi_fmac(sm[mm - 1], cphi, cm[mm - 1] * sphi);
  }
  // rotation about y by -theta: cos = ct, sin = -st
  DMats<T> dm;
  gbi_dmat1<T>(ct, -st, dm.d1);
  if constexpr (MAXK >= 2) gbi_dmat2<T>(ct, -st, dm.d2);
  if constexpr (MAXK >= 3) gbi_dmat3<T>(ct, -st, dm.d3);
  if constexpr (MAXK >= 4) gbi_dmat4<T>(ct, -st, dm.d4);
  if constexpr (MAXK >= 5) gbi_dmat5<T>(ct, -st, dm.d5);
  T ep[7];
  ep[0] = T(1);
#pragma unroll
  for (int i = 1; i < 7; ++i) ep[i] = ep[i - 1] * eps;
  T xs[S::D], yy[S::D];
  to_pair_frame<TR, T, S::MC0, S::MC1>(xl, xs, cm, sm, dm, ep);
  couple<TR, ROWS, COLS, T>(e2, xs, yy);
  from_pair_frame<TR, T, S::MR0, S::MR1, S::R0>(yy, acc, cm, sm, dm, ep);
}

// FP64 form.  Block = TPB target spheres x WPT warps per target; sources are staged in
// shared-memory tiles.  The WPT warps of a target split its sources (lane-strided
// within each tile); their partial sums are combined in shared memory in a fixed order,
// so results are deterministic.  The FP64 pipe (1/64 of the FP32 rate) bounds this
// pass, so the tile bookkeeping is not what limits it.
template <int TR, int ROWS, int COLS, typename T, int TPB, int WPT, int TILE>
__global__ void __launch_bounds__(TPB * WPT * 32) pair_kernel(const PairArgs args) {
  static_assert(std::is_same<T, double>::value, "the tiled pass is the FP64 one");
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int D = S::D;
  constexpr int R0 = S::R0;
  constexpr int C0 = S::C0;
  constexpr int C1 = S::C1;
  constexpr int NR = S::NR;
  constexpr int NC = S::NC;
  constexpr int THREADS = TPB * WPT * 32;

  __shared__ double s_pos[3][TILE];
  __shared__ double s_x[NC][TILE];

  if (args.active != nullptr && *args.active == 0) return;   // device-side GMRES has stopped
  const double* __restrict__ xsrc = args.x_index ? args.x + (size_t)(*args.x_index) * args.x_stride : args.x;
  const int N = args.N;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int tgt = warp / WPT;            // target slot in the block
  const int sub = warp - tgt * WPT;      // which share of the sources
  const int n = blockIdx.x * TPB + tgt;
  // source range of this target's system (the whole set without batching)
  int src_lo = 0, src_hi = N;
  bool active = n < N;
  if (active && args.sys_of != nullptr) {
    const int sy = args.sys_of[n];
    src_lo = args.sys_off[sy];
    src_hi = args.sys_off[sy + 1];
    if (args.sys_flag != nullptr && args.sys_flag[(size_t)sy * args.sys_flag_stride] == 0) active = false;
  }
  // the block's tile range: union of its targets' ranges
  int blk_lo = 0, blk_hi = N;
  if (args.sys_of != nullptr) {
    __shared__ int s_rng[2];
    if (threadIdx.x == 0) { s_rng[0] = N; s_rng[1] = 0; }
    __syncthreads();
    if (lane == 0 && sub == 0 && active) {
      atomicMin(&s_rng[0], src_lo);
      atomicMax(&s_rng[1], src_hi);
    }
    __syncthreads();
    blk_lo = s_rng[0];
    blk_hi = s_rng[1];
  }
  const double a = args.a;

  double tp[3] = {0.0, 0.0, 0.0};
  if (active) {
    const dpos4 p = args.pos.p64[n];
    tp[0] = p.x; tp[1] = p.y; tp[2] = p.z;
  }

  double acc[NR];
#pragma unroll
  for (int p = 0; p < NR; ++p) acc[p] = 0.0;
  float min_r2 = 3.0e38f;

  for (int base = blk_lo; base < blk_hi; base += TILE) {
    const int len = min(TILE, blk_hi - base);
    __syncthreads();
    for (int idx = threadIdx.x; idx < len; idx += THREADS) {
      const dpos4 p = args.pos.p64[base + idx];
      s_pos[0][idx] = p.x; s_pos[1][idx] = p.y; s_pos[2][idx] = p.z;
    }
    // source coefficients: component-major rows, no integer division in the loop
    for (int q = 0; q < NC; ++q) {
      const double* src = xsrc + (size_t)q * N + base;
      const double cs = args.colscale[C0 + q];
      for (int j = threadIdx.x; j < len; j += THREADS) s_x[q][j] = src[j] * cs;
    }
    __syncthreads();
    if (active) {
      for (int j = sub * 32 + lane; j < len; j += WPT * 32) {
        const int m = base + j;
        if (m == n || m < src_lo || m >= src_hi) continue;
        const double dx = tp[0] - s_pos[0][j];
        const double dy = tp[1] - s_pos[1][j];
        const double dz = tp[2] - s_pos[2][j];
        min_r2 = fminf(min_r2, float(dx * dx + dy * dy + dz * dz));
        double xl[D];
#pragma unroll
        for (int q = C0; q < C1; ++q) xl[q] = s_x[q - C0][j];
        pair_body<TR, ROWS, COLS, double>(dx, dy, dz, a, xl, acc);
      }
    }
  }

  // warp reduction of the partial sums (fixed order: deterministic)
#pragma unroll
  for (int p = 0; p < NR; ++p) {
    double v = acc[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += gbi_shfl(v, o);
    acc[p] = v;
  }
  if (args.min_r2_bits != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) min_r2 = fminf(min_r2, __shfl_xor_sync(0xffffffffu, min_r2, o));
    if (active && lane == 0) atomicMin(args.min_r2_bits, __float_as_uint(min_r2));
  }
  if constexpr (WPT > 1) {
    // combine the WPT warps of each target through shared memory (reuses the tile)
    __syncthreads();
    double* red = &s_x[0][0];
    static_assert(sizeof(s_x) >= sizeof(double) * TPB * WPT * NR || NR == 0, "reduction buffer too small");
    if (lane == 0) {
#pragma unroll
      for (int p = 0; p < NR; ++p) red[(tgt * WPT + sub) * NR + p] = acc[p];
    }
    __syncthreads();
    if (sub == 0 && lane == 0) {
#pragma unroll
      for (int p = 0; p < NR; ++p) {
        double v = red[(tgt * WPT) * NR + p];
        for (int w = 1; w < WPT; ++w) v += red[(tgt * WPT + w) * NR + p];
        acc[p] = v;
      }
    }
  }
  if (active && sub == 0 && lane == 0) {
    const double inva = 1.0 / args.a;
#pragma unroll
    for (int p = 0; p < NR; ++p) {
      double v = acc[p] * inva;
      if (args.add_self) v += args.selfg[R0 + p] * inva * xsrc[(size_t)(R0 - C0 + p) * N + n] * args.colscale[R0 + p];
      double* dst = args.y + (size_t)p * N + n;
      *dst = args.alpha * v + (args.beta != 0.0 ? args.beta * (*dst) : 0.0);
    }
  }
}

// ---------------------------------------------------------------------------------
// Streaming form for the FP32 and double-float passes.
//
// Source m is one record: NCP = NC rounded up to a multiple of 4 floats holding
// float(x_m * colscale) (double-float: the hi block then the lo block), read with
// 16-byte loads through L1 (every warp on an SM walks the same sources, so they hit).
// One block per target sphere, WPT warps splitting its sources lane by lane: no
// shared-memory tiles and no block barrier inside the loop.  The per-lane partial
// sums are combined by a transposing warp reduction and then across the WPT warps in
// shared memory, both in a fixed order, so the result does not depend on timing.  For a
// single system whose blocks do not fill whole waves, the targets of the last wave may be
// split into nsplit blocks over their sources (PairArgs::split_from; off unless the caller
// asks for it), added in part order.
// ---------------------------------------------------------------------------------

template <int NC> struct RecShape {
  static constexpr int NCP = (NC + 3) & ~3;   // floats per block of a record
  static constexpr int NV = NCP / 4;          // float4 per block
};

// Component i of a float4 register array (i is a compile-time constant after unrolling).
__device__ __forceinline__ float f4c(const float4* v, int i) {
  const float4 t = v[i >> 2];
  const int c = i & 3;
  return c == 0 ? t.x : (c == 1 ? t.y : (c == 2 ? t.z : t.w));
}

// Sum NV per-lane values over the warp.  At each step a lane keeps one half of its
// values and sends the other half to its partner, so 32 values cost 31 shuffles
// instead of 160; afterwards lane L holds the total of value 32c + L in out[c].
template <typename T, int NV>
__device__ __forceinline__ void warp_transpose_sum(const T* v, T* out) {
  constexpr int NCH = (NV + 31) / 32;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < NCH; ++c) {
    T w[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) w[i] = (32 * c + i < NV) ? v[32 * c + i] : T(0);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < o; ++i) {
        const T keep = up ? w[i + o] : w[i];
        const T send = up ? w[i] : w[i + o];
        w[i] = keep + gbi_shfl(send, o);
      }
    }
    out[c] = w[0];
  }
}

// One source m (not the target) of target n, centre th + tl, in the streaming forms:
// the pair body on m's record, accumulated into acc; min_r2 keeps the smallest r^2.
template <int TR, int ROWS, int COLS, typename T>
__device__ __forceinline__ void stream_source(const PairArgs& args, const float4* __restrict__ rec, float4 th,
                                              float4 tl, int m, T a, T* acc, float& min_r2) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int D = S::D;
  constexpr int C0 = S::C0;
  constexpr int NC = S::NC;
  constexpr bool DF = std::is_same<T, df>::value;
  constexpr int NCP = RecShape<NC>::NCP;
  constexpr int NV = RecShape<NC>::NV;
  constexpr int RECV = DF ? 2 * NV : NV;
  const float4 sh = __ldg(args.pos.hi + m), sl = __ldg(args.pos.lo + m);
  float4 r4[RECV];
#pragma unroll
  for (int i = 0; i < RECV; ++i) r4[i] = __ldg(rec + (size_t)m * RECV + i);
  T dx, dy, dz;
  if constexpr (DF) {
    // exact difference of the hi parts, plus the (tiny) difference of the lo parts
    dx = df_two_sum(th.x, -sh.x) + df(tl.x - sl.x, 0.f);
    dy = df_two_sum(th.y, -sh.y) + df(tl.y - sl.y, 0.f);
    dz = df_two_sum(th.z, -sh.z) + df(tl.z - sl.z, 0.f);
  } else {
    dx = (th.x - sh.x) + (tl.x - sl.x);
    dy = (th.y - sh.y) + (tl.y - sl.y);
    dz = (th.z - sh.z) + (tl.z - sl.z);
  }
  min_r2 = fminf(min_r2, float(dx * dx + dy * dy + dz * dz));
  T xl[D];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    if constexpr (DF) xl[C0 + q] = df(f4c(r4, q), f4c(r4, NCP + q));
    else xl[C0 + q] = f4c(r4, q);
  }
  pair_body<TR, ROWS, COLS, T>(dx, dy, dz, a, xl, acc);
}

// Row p (counted from the pass's first row) of target n in the streaming forms: the
// pair sum (units 1/a), the self term, then y = alpha v + beta y.
template <int TR, int ROWS, int COLS, typename T>
__device__ __forceinline__ void store_target(const PairArgs& args, int n, int p, double sum) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int R0 = S::R0;
  constexpr int C0 = S::C0;
  constexpr int NC = S::NC;
  constexpr bool DF = std::is_same<T, df>::value;
  constexpr int RECV = DF ? 2 * RecShape<NC>::NV : RecShape<NC>::NV;
  const double inva = 1.0 / args.a;
  double v = sum * inva;
  if (args.add_self) {
    // FP32 passes use the rounded source the pair terms saw; double-float the FP64 one
    const int q = R0 - C0 + p;
    const double* xsrc = args.x_index ? args.x + (size_t)(*args.x_index) * args.x_stride : args.x;
    const double xs = DF ? xsrc[(size_t)q * args.N + n] * args.colscale[R0 + p]
                         : double(args.x32[(size_t)n * (RECV * 4) + q]);
    v += args.selfg[R0 + p] * inva * xs;
  }
  double* dst = args.y + (size_t)p * args.N + n;
  *dst = args.alpha * v + (args.beta != 0.0 ? args.beta * (*dst) : 0.0);
}

template <int TR, int ROWS, int COLS, typename T, int WPT, int MINB>
__global__ void __launch_bounds__(WPT * 32, MINB) pair_stream_kernel(const PairArgs args) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int NR = S::NR;
  constexpr bool DF = std::is_same<T, df>::value;
  static_assert(DF || std::is_same<T, float>::value, "streaming pass is FP32 or double-float");
  constexpr int NRC = (NR + 31) / 32;
  __shared__ T red[WPT > 1 ? WPT : 1][NRC * 32];

  pdl_wait();
  if (args.active != nullptr && *args.active == 0) return;   // device-side GMRES has stopped
  // block -> target n and, for the split tail, which part of its sources
  int n = blockIdx.x, part = 0, nparts = 1;
  if (args.nsplit > 1 && n >= args.split_from) {
    const int t = n - args.split_from;
    n = args.split_from + t / args.nsplit;
    part = t - (n - args.split_from) * args.nsplit;
    nparts = args.nsplit;
  }
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  int src_lo = 0, src_hi = args.N;
  if (args.sys_of != nullptr) {
    const int sy = args.sys_of[n];
    // the whole block belongs to target n, so this return is uniform
    if (args.sys_flag != nullptr && args.sys_flag[(size_t)sy * args.sys_flag_stride] == 0) return;
    src_lo = args.sys_off[sy];
    src_hi = args.sys_off[sy + 1];
  }
  const T a = T(args.a);
  const float4 th = args.pos.hi[n], tl = args.pos.lo[n];
  const float4* __restrict__ rec = reinterpret_cast<const float4*>(args.x32);

  T acc[NR];
#pragma unroll
  for (int p = 0; p < NR; ++p) acc[p] = T(0);
  float min_r2 = 3.0e38f;

  if (nparts > 1) {
    const int len = src_hi - src_lo;
    const int lo = src_lo + (int)((long long)len * part / nparts);
    src_hi = src_lo + (int)((long long)len * (part + 1) / nparts);
    src_lo = lo;
  }
  for (int m = src_lo + warp * 32 + lane; m < src_hi; m += WPT * 32) {
    if (m == n) continue;
    stream_source<TR, ROWS, COLS, T>(args, rec, th, tl, m, a, acc, min_r2);
  }

  T tot[NRC];
  warp_transpose_sum<T, NR>(acc, tot);
  if (args.min_r2_bits != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) min_r2 = fminf(min_r2, __shfl_xor_sync(0xffffffffu, min_r2, o));
    if (lane == 0) atomicMin(args.min_r2_bits, __float_as_uint(min_r2));
  }
  if constexpr (WPT > 1) {
#pragma unroll
    for (int c = 0; c < NRC; ++c) red[warp][32 * c + lane] = tot[c];
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int c = 0; c < NRC; ++c) {
      T v = red[0][32 * c + lane];
#pragma unroll
      for (int w = 1; w < WPT; ++w) v += red[w][32 * c + lane];
      tot[c] = v;
    }
  }
  if (nparts > 1) {
    // this part's rows; the last part of the target to arrive adds all parts in order
    const int ts = n - args.split_from;
    double* slots = static_cast<double*>(args.tile_part) + (size_t)ts * nparts * (NRC * 32);
#pragma unroll
    for (int c = 0; c < NRC; ++c) slots[(size_t)part * (NRC * 32) + 32 * c + lane] = gbi_to_double(tot[c]);
    __threadfence();
    unsigned int prev = 0;
    if (lane == 0) prev = atomicAdd(args.tile_cnt + ts, 1u);
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != (unsigned int)(nparts - 1)) return;
    __threadfence();
#pragma unroll
    for (int c = 0; c < NRC; ++c) {
      double v = 0.0;
      for (int q = 0; q < nparts; ++q) v += __ldcg(slots + (size_t)q * (NRC * 32) + 32 * c + lane);
      const int p = 32 * c + lane;
      if (p < NR) store_target<TR, ROWS, COLS, T>(args, n, p, v);
    }
    if (lane == 0) args.tile_cnt[ts] = 0u;   // zero again for the next launch
    return;
  }
#pragma unroll
  for (int c = 0; c < NRC; ++c) {
    const int p = 32 * c + lane;
    if (p < NR) store_target<TR, ROWS, COLS, T>(args, n, p, gbi_to_double(tot[c]));
  }
}

}  // namespace gbi
