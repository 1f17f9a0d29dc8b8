// FP32 stage kernel for N = 4 with the symmetric volume rule and the dense
// contractions on the tensor cores (template parameter N + 8 + 32).
#define ESDG_N (4 + 8 + 32)
#define ESDG_STAGE2_ONLY
#include "esdg_kernels_impl.cuh"
