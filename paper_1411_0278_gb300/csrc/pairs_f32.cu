// FP32 instantiations of the pair operator.
#include "pairs_inst.cuh"

namespace gbi {
cudaError_t launch_pairs_f32(int trunc, int rows, int cols, const PairArgs& args, cudaStream_t stream) {
  return launch_pairs_t<float>(trunc, rows, cols, args, stream);
}
}  // namespace gbi
