// Kernel instantiations for polynomial degree N = 5.
#define ESDG_N 5
#include "esdg_kernels_impl.cuh"
