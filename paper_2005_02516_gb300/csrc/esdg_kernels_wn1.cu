// Kernel instantiations for polynomial degree N = 1 with the collapsed volume
// rule and the weight-adjusted inverse mass (template parameter N + 16).
#define ESDG_N (1 + 16)
#include "esdg_kernels_impl.cuh"
