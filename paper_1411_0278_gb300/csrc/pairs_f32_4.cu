// FP32 instantiations of the pair operator, truncation l <= 4.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f32_4, float, 4, true)
