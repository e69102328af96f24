// FP64 instantiations of the pair operator, truncation l <= 2.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f64_2, double, 2, true)
