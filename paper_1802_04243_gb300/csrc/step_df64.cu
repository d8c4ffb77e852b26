// step_df64.cu -- the persistent step kernels of a batch in double-float arithmetic
// (k_step, phase_kernels.cuh; launched by persistent.cu).
#include "phase_kernels.cuh"

STG_STEP_KERNELS(stg::PREC_DF64)
