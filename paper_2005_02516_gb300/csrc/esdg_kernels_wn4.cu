// Kernel instantiations for polynomial degree N = 4 with the collapsed volume
// rule and the weight-adjusted inverse mass (template parameter N + 16).
#define ESDG_N (4 + 16)
#include "esdg_kernels_impl.cuh"
