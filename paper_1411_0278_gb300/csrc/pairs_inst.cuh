// Instantiation and launch of the pair kernel for one arithmetic type and truncation.
#pragma once

#include "pair_chunk.cuh"
#include "pair_kernel.cuh"
#include "pair_tile.cuh"

namespace gbi {

// FULL adds the all-rows/all-columns pass (used by gbi_apply only).
template <typename T, int TRN, bool FULL>
cudaError_t launch_pairs_tt(int rows, int cols, const PairArgs& args, cudaStream_t stream) {
  if (args.N <= 0) return cudaSuccess;
  const int N = args.N;
  if constexpr (std::is_same<T, double>::value) {
    // FP64: shared-memory tiles of 64 sources; the FP64 pipe bounds this pass
    constexpr int TILE = 64;
    const int wpt = N >= 2048 ? 1 : (N >= 1024 ? 2 : 4);
#define GBI_L(RV, CV, TPB, WPT)                                                          \
  if (rows == RV && cols == CV && wpt == WPT) {                                          \
    const dim3 grid((N + TPB - 1) / TPB), block(TPB * WPT * 32);                         \
    pair_kernel<TRN, RV, CV, T, TPB, WPT, TILE><<<grid, block, 0, stream>>>(args);      \
    return cudaGetLastError();                                                           \
  }
#define GBI_LW(RV, CV) GBI_L(RV, CV, 4, 1) GBI_L(RV, CV, 2, 2) GBI_L(RV, CV, 1, 4)
    GBI_LW(SET_H, SET_L)
    GBI_LW(SET_H, SET_H)
    GBI_LW(SET_L, SET_ALL)
    if constexpr (FULL) {
      GBI_LW(SET_ALL, SET_ALL)
    }
#undef GBI_LW
#undef GBI_L
  } else {
    // at most 16 resident warps per SM for the FP32 forms of l <= 3 (a 128-register
    // cap), 8 for l <= 4 and double-float; stream_wpt keeps WPT within the same bound
    constexpr bool DF = std::is_same<T, df>::value;
    constexpr int WARPS_SM = (TRN == 4 || DF) ? 8 : 16;
    if (args.wpt == kFormChunk) {
      // chunk-balanced streaming form (pair_chunk.cuh): plan and scratch in PairArgs
#define GBI_K(RV, CV)                                                                              \
  if (rows == RV && cols == CV) {                                                                  \
    return launch_pdl(args.pdl != 0, dim3(args.tile_P), dim3(kChunkWarps * 32), stream,            \
                      pair_chunk_kernel<TRN, RV, CV, T, WARPS_SM / kChunkWarps>, args);            \
  }
      GBI_K(SET_H, SET_L)
      GBI_K(SET_H, SET_H)
      GBI_K(SET_L, SET_ALL)
      if constexpr (FULL) {
        GBI_K(SET_ALL, SET_ALL)
      }
#undef GBI_K
      return cudaErrorInvalidValue;
    }
    if (args.wpt == kFormTile) {
      // tiled form (pair_tile.cuh): the caller filled the plan and scratch of PairArgs
#define GBI_T(RV, CV)                                                                              \
  if (rows == RV && cols == CV) {                                                                  \
    constexpr size_t smem = tile_smem_bytes<TRN, RV, CV, T>();                                     \
    static bool attr = false;                                                                      \
    if (!attr) {                                                                                   \
      const cudaError_t ea = cudaFuncSetAttribute(pair_tile_kernel<TRN, RV, CV, T>,                \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                                  int(smem));                                      \
      if (ea != cudaSuccess) return ea;                                                            \
      attr = true;                                                                                 \
    }                                                                                              \
    return launch_pdl_smem(args.pdl != 0, dim3(args.tile_P), dim3(TileShape<T, TRN>::WARPS * 32), smem, \
                           stream, pair_tile_kernel<TRN, RV, CV, T>, args);                        \
  }
      GBI_T(SET_H, SET_L)
      GBI_T(SET_H, SET_H)
      GBI_T(SET_L, SET_ALL)
      if constexpr (FULL) {
        GBI_T(SET_ALL, SET_ALL)
      }
#undef GBI_T
      return cudaErrorInvalidValue;
    }
    const int wpt = stream_wpt(TRN, DF ? 2 : 1, N, args.wpt);
#define GBI_S(RV, CV, WPT)                                                                         \
  if (rows == RV && cols == CV && wpt == WPT) {                                                    \
    constexpr int MINB = WARPS_SM / WPT > 0 ? WARPS_SM / WPT : 1;                                  \
    const int blocks = (args.nsplit > 1 && args.split_from < N) ? args.split_from + (N - args.split_from) * args.nsplit : N; \
    return launch_pdl(args.pdl != 0, dim3(blocks), dim3(WPT * 32), stream,                         \
                      pair_stream_kernel<TRN, RV, CV, T, WPT, MINB>, args);                        \
  }
#define GBI_SW(RV, CV) \
  GBI_S(RV, CV, 2) GBI_S(RV, CV, 4) GBI_S(RV, CV, 8) if constexpr (WARPS_SM >= 16) { GBI_S(RV, CV, 16) }
    GBI_SW(SET_H, SET_L)
    GBI_SW(SET_H, SET_H)
    GBI_SW(SET_L, SET_ALL)
    if constexpr (FULL) {
      GBI_SW(SET_ALL, SET_ALL)
    }
#undef GBI_SW
#undef GBI_S
  }
  return cudaErrorInvalidValue;
}

}  // namespace gbi

#define GBI_PAIRS_TU(NAME, T, TRN, FULL)                                                         \
  namespace gbi {                                                                                \
  cudaError_t NAME(int rows, int cols, const PairArgs& args, cudaStream_t stream) {              \
    return launch_pairs_tt<T, TRN, FULL>(rows, cols, args, stream);                             \
  }                                                                                              \
  }
