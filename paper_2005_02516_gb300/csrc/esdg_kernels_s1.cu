// Kernel instantiations for polynomial degree N = 1 with the symmetric
// volume rule (template parameter N + 8).
#define ESDG_N (1 + 8)
#include "esdg_kernels_impl.cuh"
