// FP32 instantiations of the pair operator, truncation l <= 2.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f32_2, float, 2, true)
