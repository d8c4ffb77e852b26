// phase_df64.cu -- the equation kernels of one loop-2 iteration in
// double-float arithmetic (float pairs on the FP32 pipe; phase_kernels.cuh).
#include "phase_kernels.cuh"

STG_PHASE_LAUNCHERS(stg::PREC_DF64)
