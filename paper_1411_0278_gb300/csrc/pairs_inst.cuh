// Instantiation and launch of the pair kernel for one arithmetic type.
#pragma once

#include "pair_kernel.cuh"

namespace gbi {

template <typename T>
cudaError_t launch_pairs_t(int trunc, int rows, int cols, const PairArgs& args, cudaStream_t stream) {
  constexpr int WARPS = 4;
  constexpr int TILE = sizeof(T) == 4 ? 128 : 64;
  if (args.N <= 0) return cudaSuccess;
  const dim3 grid((args.N + WARPS - 1) / WARPS), block(WARPS * 32);
#define GBI_L(TRN, RV, CV)                                                              \
  if (trunc == TRN && rows == RV && cols == CV) {                                       \
    pair_kernel<TRN, RV, CV, T, WARPS, TILE><<<grid, block, 0, stream>>>(args);        \
    return cudaGetLastError();                                                          \
  }
#define GBI_L4(TRN) GBI_L(TRN, SET_H, SET_L) GBI_L(TRN, SET_H, SET_H) GBI_L(TRN, SET_L, SET_ALL) \
  GBI_L(TRN, SET_ALL, SET_ALL)
  GBI_L4(2)
  GBI_L4(3)
  GBI_L4(4)
#undef GBI_L4
#undef GBI_L
  return cudaErrorInvalidValue;
}

}  // namespace gbi
