// DG-SBP kernels with an FP32 right-hand side (FP64 state and RK update).
#define ESDG_SBP_REAL float
#include "esdg_sbp_impl.cuh"
