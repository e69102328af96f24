// Chunk-balanced streaming form of the FP32 / double-float pair passes (the pair operator
// of Sec. III, Eq. single_layer_yl_matrix_element, as in pair_kernel.cuh), one system.
//
// The per-pair work is the streaming form's: lanes are sources, a warp accumulates the
// rows of one target over 32 sources at a time.  What changes is the partition.  The
// sources of target n, m != n in index order, form cpt = ceil((N - 1) / 32) chunks of 32;
// the N cpt chunks, target-major, are split into G contiguous, equal (to one chunk)
// ranges, one per warp of a grid of exactly the resident warps (4-warp blocks, as many
// as the SMs hold at once).  So every SM does the same number of pair evaluations and
// no partly empty last wave remains, whatever N is; a warp's range crosses a target
// boundary at most a few times.
//
// At the end of each target in its range a warp sums its lanes (the transposing warp
// reduction of the streaming form).  A target covered by one warp is stored directly.
// Otherwise the warp writes its partial rows to slot (n, k) of global scratch, k its
// position among the warps that cover n, and counts itself in n's arrival counter; the
// last to arrive adds the slots in k order and stores the result, so the sums do not
// depend on timing, and resets the counter (zero between launches).  Nothing waits on
// another warp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pair_kernel.cuh"

namespace gbi {

constexpr int kChunkWarps = 4;   // warps per block of the chunk-balanced form

struct ChunkPlan {
  int P = 0;        // blocks (kChunkWarps warps each)
  int G = 0;        // warps
  int maxseg = 0;   // warps that can cover one target (partial slots per target)
};

// warps_sm: resident warps per SM of the pass (16 for FP32 at l <= 3, else 8)
inline ChunkPlan chunk_plan(int N, int num_sms, int warps_sm) {
  ChunkPlan c;
  if (N <= 1 || num_sms <= 0) return c;
  c.P = num_sms * (warps_sm / kChunkWarps);
  c.G = c.P * kChunkWarps;
  const long long cpt = (N - 1 + 31) / 32;
  const long long C = (long long)N * cpt;
  // warps beyond the chunk count stay idle: every working warp gets per or per + 1 chunks
  const long long per = C / (c.G < C ? c.G : C);
  long long ms = (cpt + per - 1) / per + 1;
  if (ms > cpt) ms = cpt;
  c.maxseg = int(ms);
  return c;
}

inline int chunk_warps_sm(int trunc, int precision) { return (trunc == 4 || precision == 2) ? 8 : 16; }

inline size_t chunk_part_bytes(const ChunkPlan& c, int N, int nr, size_t tsize) {
  return (size_t)N * c.maxseg * (size_t)((nr + 31) / 32) * 32 * tsize;
}

#ifdef __CUDACC__
// the warp whose range holds chunk c: the largest w with floor(w C / G) <= c
__device__ __forceinline__ long long chunk_warp_of(long long c, long long C, long long G) {
  return ((c + 1) * G + C - 1) / C - 1;
}

__device__ __forceinline__ float chunk_ldcg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ df chunk_ldcg(const df* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

// End of target n in warp g's range: sum the lanes, then store, or hand over to the
// last of n's warps.
template <int TR, int ROWS, int COLS, typename T>
__device__ __forceinline__ void chunk_flush(const PairArgs& args, int n, long long g, int cpt, long long C,
                                            long long G, const T* acc) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int NR = S::NR;
  constexpr int NRC = (NR + 31) / 32;
  const int lane = threadIdx.x & 31;
  T tot[NRC];
  warp_transpose_sum<T, NR>(acc, tot);
  const long long gf = chunk_warp_of((long long)n * cpt, C, G);
  const long long gl = chunk_warp_of((long long)n * cpt + cpt - 1, C, G);
  const int nseg = int(gl - gf + 1);
  if (nseg > 1) {
    T* slots = reinterpret_cast<T*>(args.tile_part) + (size_t)n * args.tile_maxseg * (NRC * 32);
#pragma unroll
    for (int c = 0; c < NRC; ++c) slots[(size_t)(g - gf) * (NRC * 32) + 32 * c + lane] = tot[c];
    __threadfence();
    __syncwarp();
    unsigned int last = 0;
    if (lane == 0) last = atomicAdd(args.tile_cnt + n, 1u) == (unsigned int)(nseg - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int c = 0; c < NRC; ++c) {
      T v = chunk_ldcg(slots + 32 * c + lane);
      for (int k = 1; k < nseg; ++k) v = v + chunk_ldcg(slots + (size_t)k * (NRC * 32) + 32 * c + lane);
      tot[c] = v;
    }
    if (lane == 0) args.tile_cnt[n] = 0u;
  }
#pragma unroll
  for (int c = 0; c < NRC; ++c) {
    const int p = 32 * c + lane;
    if (p < NR) store_target<TR, ROWS, COLS, T>(args, n, p, gbi_to_double(tot[c]));
  }
}

template <int TR, int ROWS, int COLS, typename T, int MINB>
__global__ void __launch_bounds__(kChunkWarps * 32, MINB) pair_chunk_kernel(const PairArgs args) {
  using S = PassShape<TR, ROWS, COLS>;
  constexpr int NR = S::NR;
  static_assert(std::is_same<T, float>::value || std::is_same<T, df>::value,
                "the chunk-balanced pass is FP32 or double-float");
  pdl_wait();
  if (args.active != nullptr && *args.active == 0) return;   // device-side GMRES has stopped
  const int N = args.N;
  const int lane = threadIdx.x & 31;
  const int cpt = (N - 1 + 31) >> 5;
  const long long C = (long long)N * cpt;
  // working warps: at most one per chunk, so that every one of them has a chunk
  const long long G = args.tile_G < C ? args.tile_G : C;
  const long long g = (long long)blockIdx.x * kChunkWarps + (threadIdx.x >> 5);
  const long long c0 = g < G ? g * C / G : C, c1 = g < G ? (g + 1) * C / G : C;
  float min_r2 = 3.0e38f;
  if (c0 < c1) {
    const T a = T(args.a);
    const float4* __restrict__ rec = reinterpret_cast<const float4*>(args.x32);
    // target n and its chunk k, advanced without divisions inside the loop
    int n = int(c0 / cpt);
    int k = int(c0 - (long long)n * cpt);
    const int nchunks = int(c1 - c0);
    float4 th = args.pos.hi[n], tl = args.pos.lo[n];
    T acc[NR];
#pragma unroll
    for (int p = 0; p < NR; ++p) acc[p] = T(0);
    for (int i = 0; i < nchunks; ++i, ++k) {
      if (k == cpt) {
        chunk_flush<TR, ROWS, COLS, T>(args, n, g, cpt, C, G, acc);
        ++n;
        k = 0;
        th = args.pos.hi[n];
        tl = args.pos.lo[n];
#pragma unroll
        for (int p = 0; p < NR; ++p) acc[p] = T(0);
      }
      // source index j of target n (its own index skipped)
      const int j = k * 32 + lane;
      if (j < N - 1) stream_source<TR, ROWS, COLS, T>(args, rec, th, tl, j < n ? j : j + 1, a, acc, min_r2);
    }
    chunk_flush<TR, ROWS, COLS, T>(args, n, g, cpt, C, G, acc);
  }
  if (args.min_r2_bits != nullptr) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) min_r2 = fminf(min_r2, __shfl_xor_sync(0xffffffffu, min_r2, o));
    if (lane == 0 && min_r2 < 3.0e38f) atomicMin(args.min_r2_bits, __float_as_uint(min_r2));
  }
}
#endif

}  // namespace gbi
