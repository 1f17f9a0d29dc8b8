// Kernel instantiations for polynomial degree N = 1.
#define ESDG_N 1
#include "esdg_kernels_impl.cuh"
