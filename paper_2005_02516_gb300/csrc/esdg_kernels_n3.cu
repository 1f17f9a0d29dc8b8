// Kernel instantiations for polynomial degree N = 3.
#define ESDG_N 3
#include "esdg_kernels_impl.cuh"
