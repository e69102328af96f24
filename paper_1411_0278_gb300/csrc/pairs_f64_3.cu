// FP64 instantiations of the pair operator, truncation l <= 3.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f64_3, double, 3, true)
