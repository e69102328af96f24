// FP64 instantiations of the pair operator, truncation l <= 5 (83 components per sphere).
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f64_5, double, 5, true)
