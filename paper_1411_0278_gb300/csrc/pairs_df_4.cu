// double-float (FP32-pipe, ~48-bit) instantiations of the pair operator, truncation l <= 4.
#include "pairs_inst.cuh"

GBI_PAIRS_TU(launch_pairs_df_4, df, 4, false)
