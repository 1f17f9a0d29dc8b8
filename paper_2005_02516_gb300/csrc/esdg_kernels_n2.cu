// Kernel instantiations for polynomial degree N = 2.
#define ESDG_N 2
#include "esdg_kernels_impl.cuh"
