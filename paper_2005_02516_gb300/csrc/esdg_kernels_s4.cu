// Kernel instantiations for polynomial degree N = 4 with the symmetric
// volume rule (template parameter N + 8).
#define ESDG_N (4 + 8)
#include "esdg_kernels_impl.cuh"
