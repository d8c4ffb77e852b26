// phase_fp64.cu -- the equation kernels of one loop-2 iteration in FP64
// arithmetic, the paper's (phase_kernels.cuh).
#include "phase_kernels.cuh"

STG_PHASE_LAUNCHERS(stg::PREC_FP64)
