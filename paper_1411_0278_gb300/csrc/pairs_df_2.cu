// double-float (FP32-pipe, ~48-bit) instantiations of the pair operator, truncation l <= 2.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_df_2, df, 2, false)
