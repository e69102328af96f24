// FP32 instantiations of the pair operator, truncation l <= 3.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f32_3, float, 3, true)
