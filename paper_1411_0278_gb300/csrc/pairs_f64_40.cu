// FP64 instantiations of the pair operator, the minimal truncation of Sec. IV: every
// mode of rank <= 4 (l <= 4 without 5t, 47 components per sphere).
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_f64_40, double, 40, true)
