// Kernel instantiations for polynomial degree N = 2 with the collapsed volume
// rule and the weight-adjusted inverse mass (template parameter N + 16).
#define ESDG_N (2 + 16)
#include "esdg_kernels_impl.cuh"
