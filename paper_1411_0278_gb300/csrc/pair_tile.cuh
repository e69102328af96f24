// Tiled form of the FP32 / double-float pair passes (the pair operator of
// Sec. III, Eq. single_layer_yl_matrix_element, as in pair_kernel.cuh).
//
// Lanes are targets: a warp holds 32 consecutive target spheres (a "group") and walks
// source spheres that every lane reads at the same shared-memory address (broadcast),
// so a source record costs one load per warp instead of one per lane and no lane
// waits on a global-memory miss.  Each warp stages its own sources in shared memory
// with the TMA unit (cp.async.bulk into a two-stage ring per warp, completion through
// an mbarrier), one tile ahead of its computation, so warps never wait for each other
// inside the pair loop.
//
// Work partition: the (group, source) units, group-major, are split into P equal
// contiguous ranges, one per block (P = SMs x blocks per SM), so every SM gets the
// same number of pair evaluations whatever N is (no partly empty last wave).  A
// block's range crosses a few groups ("segments"); within a segment the warps split
// the block's sources evenly, and at its end the block sums its warps' partial sums in
// a fixed order and writes one partial row block to global scratch.  The last block to
// finish a group (an arrival counter per group) adds that group's partials in block
// order and stores the result, so the sums do not depend on timing.  That block resets
// the counter, which keeps it zero between launches.
//
// Every mbarrier wait is bounded (PairArgs::wait_limit try_wait rounds): if one gives
// up, the block agrees on it at the end of the segment, sets *err, each warp's lane 0
// waits (bounded again, with the full limit) for its copies still in flight, and the
// block returns.  The host reads *err after the solve and reports GBI_ERR_TIMEOUT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pair_kernel.cuh"

namespace gbi {

constexpr int kTileSrc = 16;                  // sources per shared-memory stage of one warp
constexpr long long kTileWaitLimit = 1ll << 24;   // try_wait rounds before giving up

// Warps per block and blocks per SM of the tiled pass: 16 warps (one block) for the
// FP32 forms of l <= 3 (128 registers each); 8 warps for l <= 4 and double-float.
template <typename T, int TR> struct TileShape {
  static constexpr bool HEAVY = TR == 4 || !std::is_same<T, float>::value;
  static constexpr int WARPS = HEAVY ? 8 : 16;
  static constexpr int BPS = 1;
};

// Dynamic shared memory of the tiled pass: the cross-warp reduction buffer, two stages
// of (records, hi, lo) per warp, the warps' mbarriers and producer states, a flag.
template <int TR, int ROWS, int COLS, typename T>
__host__ __device__ constexpr size_t tile_smem_bytes() {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr bool DF = std::is_same<T, df>::value;
  constexpr int RECV = DF ? 2 * RecShape<S::NC>::NV : RecShape<S::NC>::NV;
  constexpr int W = TileShape<T, TR>::WARPS;
  return size_t(W) * S::NR * 32 * sizeof(T) + size_t(W) * 2 * kTileSrc * (RECV + 2) * 16 + size_t(W) * 16 +
         size_t(W) * 16 + 16;
}

// Host-side plan of a tiled launch.
struct TilePlan {
  int P = 0;        // blocks
  int G = 0;        // target groups of 32
  int maxseg = 0;   // groups a block's range can touch (partial slots per block)
};

inline TilePlan tile_plan(int N, int num_sms, int bps) {
  TilePlan t;
  if (N <= 1) return t;
  t.G = (N + 31) / 32;
  const long long U = (long long)t.G * N;
  long long P = (long long)num_sms * bps;
  if (P > U / 32) P = U / 32;   // at least 32 units per block (no block is empty)
  if (P < 1) P = 1;
  t.P = int(P);
  int mx = 1;
  for (long long b = 0; b < P; ++b) {
    const long long u0 = U * b / P, u1 = U * (b + 1) / P;
    const int segs = int((u1 - 1) / N - u0 / N + 1);
    if (segs > mx) mx = segs;
  }
  t.maxseg = mx;
  return t;
}

// Scratch bytes of a plan: partial row blocks (NR x 32 values of T per slot) followed
// by one arrival counter per group.
inline size_t tile_part_bytes(const TilePlan& t, int nr, size_t tsize) {
  return (size_t)t.P * t.maxseg * nr * 32 * tsize;
}

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t tile_saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool tile_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier; false if `limit` rounds ran out.
__device__ __forceinline__ bool tile_wait(uint32_t mbar, uint32_t parity, long long limit) {
  for (long long it = 0; it < limit; ++it)
    if (tile_try_wait(mbar, parity)) return true;
  return false;
}

// Block of the unit range containing unit x: the largest b with floor(U b / P) <= x.
__device__ __forceinline__ int tile_block_of(long long x, long long U, int P) {
  return int(((x + 1) * P + U - 1) / U) - 1;
}

// partial sums written by other blocks: read through L2 only
__device__ __forceinline__ float tile_ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ df tile_ldcg(const df* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

template <int TR, int ROWS, int COLS, typename T>
__device__ __forceinline__ void tile_source(const float4* __restrict__ srec, const float4* __restrict__ shi,
                                            const float4* __restrict__ slo, int j, float4 th, float4 tl, T a,
                                            T* acc, float& min_r2) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int D = S::D;
  constexpr int C0 = S::C0;
  constexpr int NC = S::NC;
  constexpr bool DF = std::is_same<T, df>::value;
  constexpr int NCP = RecShape<NC>::NCP;
  constexpr int NV = RecShape<NC>::NV;
  constexpr int RECV = DF ? 2 * NV : NV;
  const float4 sh = shi[j], sl = slo[j];
  float4 r4[RECV];
#pragma unroll
  for (int i = 0; i < RECV; ++i) r4[i] = srec[j * RECV + i];
  T dx, dy, dz;
  if constexpr (DF) {
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

// One warp's share of segment k of a block (units [u0, u1), first group g0): the
// sources [a, b) of group g0 + k, split evenly over the WARPS warps.
__device__ __forceinline__ void tile_share(long long u0, long long u1, int N, int g0, int k, int w, int warps,
                                           int& a, int& b) {
  const long long gb = (long long)(g0 + k) * N;
  const int lo = int((u0 > gb ? u0 : gb) - gb);
  const int hi = int((u1 < gb + N ? u1 : gb + N) - gb);
  a = lo + (hi - lo) * w / warps;
  b = lo + (hi - lo) * (w + 1) / warps;
}

// Producer state of one warp (touched by its lane 0 only): the next tile to issue, as
// (segment, first source), and the number of tiles issued so far.
struct TileProd {
  int k, pos, issued, pad;
};

template <int TR, int ROWS, int COLS, typename T>
__global__ void __launch_bounds__(TileShape<T, TR>::WARPS * 32, TileShape<T, TR>::BPS)
    pair_tile_kernel(const PairArgs args) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int NR = S::NR;
  constexpr int NC = S::NC;
  constexpr bool DF = std::is_same<T, df>::value;
  static_assert(DF || std::is_same<T, float>::value, "tiled pass is FP32 or double-float");
  constexpr int WARPS = TileShape<T, TR>::WARPS;
  constexpr int THREADS = WARPS * 32;
  constexpr int RECV = DF ? 2 * RecShape<NC>::NV : RecShape<NC>::NV;
  constexpr int TW = kTileSrc;                  // sources per warp stage
  constexpr int STAGE_V = TW * (RECV + 2);      // float4 per warp stage

  extern __shared__ __align__(128) unsigned char tile_smem[];
  T* red = reinterpret_cast<T*>(tile_smem);
  float4* stages = reinterpret_cast<float4*>(tile_smem + size_t(WARPS) * NR * 32 * sizeof(T));
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(stages + size_t(WARPS) * 2 * STAGE_V);
  TileProd* prod = reinterpret_cast<TileProd*>(mbar + 2 * WARPS);
  int* s_flag = reinterpret_cast<int*>(prod + WARPS);

  pdl_wait();
  if (args.active != nullptr && *args.active == 0) return;   // device-side GMRES has stopped
  // one system: every target belongs to system 0, whose flag stops the whole pass
  if (args.sys_flag != nullptr && args.sys_flag[0] == 0) return;
  const int N = args.N;
  const int P = args.tile_P;
  const long long U = (long long)args.tile_G * N;
  const long long u0 = U * blockIdx.x / P, u1 = U * (blockIdx.x + 1) / P;
  if (u0 >= u1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g0 = int(u0 / N);
  const int nseg = int((u1 - 1) / N) - g0 + 1;
  float4* wst = stages + size_t(warp) * 2 * STAGE_V;   // this warp's two stages
  const uint32_t mb0 = tile_saddr(&mbar[2 * warp]), mb1 = tile_saddr(&mbar[2 * warp + 1]);

  // lane 0: issue the warp's next tile (if any) into stage issued & 1
  auto issue = [&]() {
    TileProd pr = prod[warp];
    if (pr.k >= nseg) return;
    int a, b;
    tile_share(u0, u1, N, g0, pr.k, warp, WARPS, a, b);
    while (pr.pos >= b) {
      if (++pr.k >= nseg) {
        prod[warp] = pr;
        return;
      }
      tile_share(u0, u1, N, g0, pr.k, warp, WARPS, a, b);
      pr.pos = a;
    }
    const int m0 = pr.pos;
    const int len = min(TW, b - m0);
    float4* dst = wst + (pr.issued & 1) * STAGE_V;
    const uint32_t mb = (pr.issued & 1) ? mb1 : mb0;
    const uint32_t bytes = uint32_t(len) * uint32_t(RECV * 16 + 32);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tile_saddr(dst)),
        "l"(reinterpret_cast<const float4*>(args.x32) + (size_t)m0 * RECV), "r"(uint32_t(len * RECV * 16)), "r"(mb)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tile_saddr(dst + TW * RECV)),
        "l"(args.pos.hi + m0), "r"(uint32_t(len * 16)), "r"(mb)
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            tile_saddr(dst + TW * (RECV + 1))),
        "l"(args.pos.lo + m0), "r"(uint32_t(len * 16)), "r"(mb)
        : "memory");
    pr.pos = m0 + len;
    ++pr.issued;
    prod[warp] = pr;
  };

  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb0), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mb1), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    int a, b;
    tile_share(u0, u1, N, g0, 0, warp, WARPS, a, b);
    prod[warp] = TileProd{0, a, 0, 0};
    issue();
    issue();
  }
  __syncwarp();

  const T a = T(args.a);
  int t = 0;          // tiles this warp has consumed
  bool bad = false;   // a stage wait gave up
  for (int k = 0; k < nseg; ++k) {
    const int g = g0 + k;
    const int n = g * 32 + lane;
    const float4 th = args.pos.hi[min(n, N - 1)], tl = args.pos.lo[min(n, N - 1)];
    T acc[NR];
#pragma unroll
    for (int p = 0; p < NR; ++p) acc[p] = T(0);
    float min_r2 = 3.0e38f;
    int sa, sb;
    tile_share(u0, u1, N, g0, k, warp, WARPS, sa, sb);
    for (int pos = sa; pos < sb && !bad; pos += TW, ++t) {
      const int len = min(TW, sb - pos);
      const uint32_t mb = (t & 1) ? mb1 : mb0;
      if (!tile_wait(mb, uint32_t((t >> 1) & 1), args.wait_limit)) {
        bad = true;
        break;
      }
      const float4* srec = wst + (t & 1) * STAGE_V;
      const float4* shi = srec + TW * RECV;
      const float4* slo = shi + TW;
      if (n < N) {
        for (int j = 0; j < len; ++j) {
          if (pos + j == n) continue;
          tile_source<TR, ROWS, COLS, T>(srec, shi, slo, j, th, tl, a, acc, min_r2);
        }
      }
      __syncwarp();   // the whole warp is done with this stage
      if (lane == 0) issue();
    }
    // this block's share of group g: warps in a fixed order, then one partial block
#pragma unroll
    for (int p = 0; p < NR; ++p) red[(warp * NR + p) * 32 + lane] = acc[p];
    if (__syncthreads_or(bad)) {
      // a stage did not arrive in time: record it; lane 0 of every warp waits (bounded
      // again, with the full limit) for its copies still in flight before the block exits
      if (lane == 0) {
        if (tid == 0 && args.err != nullptr) atomicExch(args.err, 1);
        const int issued = prod[warp].issued;
        for (int q = t; q < issued; ++q) tile_wait((q & 1) ? mb1 : mb0, uint32_t((q >> 1) & 1), kTileWaitLimit);
      }
      return;
    }
    T* part = reinterpret_cast<T*>(args.tile_part) + ((size_t)blockIdx.x * args.tile_maxseg + k) * (NR * 32);
    for (int o = tid; o < NR * 32; o += THREADS) {
      T v = red[o];
#pragma unroll
      for (int w = 1; w < WARPS; ++w) v += red[w * NR * 32 + o];
      part[o] = v;
    }
    if (args.min_r2_bits != nullptr) {
      float mr = n < N ? min_r2 : 3.0e38f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mr = fminf(mr, __shfl_xor_sync(0xffffffffu, mr, o));
      if (lane == 0) atomicMin(args.min_r2_bits, __float_as_uint(mr));
    }
    __threadfence();
    __syncthreads();
    const long long gu0 = (long long)g * N;
    const int b0 = tile_block_of(gu0, U, P), b1 = tile_block_of(gu0 + N - 1, U, P);
    if (tid == 0) {
      const unsigned int prev = atomicAdd(args.tile_cnt + g, 1u);
      *s_flag = prev == unsigned(b1 - b0);
    }
    __syncthreads();
    if (*s_flag) {
      // last arrival: add the group's partials in block order (loads of up to eight
      // blocks in flight at once) and store
      __threadfence();
      for (int o = tid; o < NR * 32; o += THREADS) {
        T v = T(0);
        for (int bb = b0; bb <= b1; bb += 8) {
          T pv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int b = bb + i;
            if (b <= b1) {
              const int gf = int((U * b / P) / N);
              pv[i] = tile_ldcg(reinterpret_cast<const T*>(args.tile_part) +
                                ((size_t)b * args.tile_maxseg + (g - gf)) * (NR * 32) + o);
            }
          }
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (bb + i <= b1) v = (bb + i == b0) ? pv[i] : v + pv[i];
        }
        const int nn = g * 32 + (o & 31);
        if (nn < N) store_target<TR, ROWS, COLS, T>(args, nn, o >> 5, gbi_to_double(v));
      }
      if (tid == 0) args.tile_cnt[g] = 0u;
    }
    __syncthreads();   // red and s_flag are reused by the next segment
  }
}

#endif

}  // namespace gbi
