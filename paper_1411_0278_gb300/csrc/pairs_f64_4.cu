// FP64 instantiations of the pair operator, truncation l <= 4.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f64_4, double, 4, true)
