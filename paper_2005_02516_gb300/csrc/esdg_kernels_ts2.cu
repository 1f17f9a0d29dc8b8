// FP32 stage kernel for N = 2 with the symmetric volume rule and the dense
// contractions on the tensor cores (template parameter N + 8 + 32).
#define ESDG_N (2 + 8 + 32)
#define ESDG_STAGE2_ONLY
#include "esdg_kernels_impl.cuh"
