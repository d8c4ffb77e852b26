// step_mixed.cu -- the persistent step kernels of a batch in the mixed path's arithmetic
// (FP32 assembly; FP64 pressure, equation of state and residuals)
// (k_step, phase_kernels.cuh; launched by persistent.cu).
#include "phase_kernels.cuh"

STG_STEP_KERNELS(stg::PREC_MIXED)
