// double-float (FP32-pipe, ~48-bit) instantiations of the pair operator, truncation l <= 3.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_df_3, df, 3, false)
