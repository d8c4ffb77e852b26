// step_fp64.cu -- the persistent step kernels of a batch in FP64 arithmetic, the paper's
// (k_step, phase_kernels.cuh; launched by persistent.cu).
#include "phase_kernels.cuh"

STG_STEP_KERNELS(stg::PREC_FP64)
