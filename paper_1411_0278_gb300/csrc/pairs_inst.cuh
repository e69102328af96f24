// Instantiation and launch of the pair kernel for one arithmetic type and truncation.
#pragma once

#include "pair_kernel.cuh"

namespace gbi {

// Warps per target chosen so that about 2400 warps (one wave at 16 resident warps per
// SM on 152 SMs) exist when N is small; blocks stay at four warps.  FULL adds the
// all-rows/all-columns pass (used by gbi_apply only).
template <typename T, int TRN, bool FULL>
cudaError_t launch_pairs_tt(int rows, int cols, const PairArgs& args, cudaStream_t stream) {
  constexpr int TILE = sizeof(T) == 4 ? 128 : 64;   // 64 for double and double-float
  if (args.N <= 0) return cudaSuccess;
  const int N = args.N;
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
  return cudaErrorInvalidValue;
}

}  // namespace gbi

#define GBI_PAIRS_TU(NAME, T, TRN, FULL)                                                         \
  namespace gbi {                                                                                \
  cudaError_t NAME(int rows, int cols, const PairArgs& args, cudaStream_t stream) {              \
    return launch_pairs_tt<T, TRN, FULL>(rows, cols, args, stream);                             \
  }                                                                                              \
  }
