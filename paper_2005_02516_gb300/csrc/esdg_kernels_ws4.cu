// Kernel instantiations for polynomial degree N = 4 with the symmetric volume
// rule and the weight-adjusted inverse mass (template parameter N + 8 + 16).
#define ESDG_N (4 + 8 + 16)
#include "esdg_kernels_impl.cuh"
