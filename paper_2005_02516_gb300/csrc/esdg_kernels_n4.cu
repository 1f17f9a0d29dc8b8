// Kernel instantiations for polynomial degree N = 4.
#define ESDG_N 4
#include "esdg_kernels_impl.cuh"
