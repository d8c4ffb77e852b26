// phase_mixed.cu -- the equation kernels of one loop-2 iteration in the mixed
// path: FP32 assembly, FP64 pressure, equation of state and residuals
// (phase_kernels.cuh).
#include "phase_kernels.cuh"

STG_PHASE_LAUNCHERS(stg::PREC_MIXED)
