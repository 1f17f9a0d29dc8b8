// Kernel instantiations for polynomial degree N = 3 with the symmetric
// volume rule (template parameter N + 8).
#define ESDG_N (3 + 8)
#include "esdg_kernels_impl.cuh"
