// Kernel instantiations for polynomial degree N = 2 with the symmetric
// volume rule (template parameter N + 8).
#define ESDG_N (2 + 8)
#include "esdg_kernels_impl.cuh"
