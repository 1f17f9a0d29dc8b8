// FP32 stage kernel for N = 1 with the symmetric volume rule and the dense
// contractions on the tensor cores (template parameter N + 8 + 32).
#define ESDG_N (1 + 8 + 32)
#define ESDG_STAGE2_ONLY
#include "esdg_kernels_impl.cuh"
