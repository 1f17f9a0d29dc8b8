// Host-side launch wrappers, one explicit instantiation per degree N (the
// esdg_kernels_nK.cu translation units compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "esdg_kernels.cuh"

namespace esdg {

// Launch geometry of the persistent stage kernels for degree N and type real:
// CTAs of 8 warps (one element per warp), as many CTAs per SM as fit.
struct LaunchGeom {
    int block = 256;
    int grid = 0;
    size_t smem = 0;
};

template <int N, typename real>
cudaError_t stage_geometry(int num_sms, LaunchGeom& lg);
template <int N, typename real>
cudaError_t launch_project(const StageParams<real>& p, const LaunchGeom& lg, cudaStream_t s);
template <int N, typename real>
cudaError_t launch_stage(const StageParams<real>& p, int mode, const LaunchGeom& lg, cudaStream_t s);
template <int N>
cudaError_t launch_entropy(int K, double g, const double* u, const double* rhs, const double* Vq, const double* wJq,
                           const double* bq, double* partial, int nparts, double* out, cudaStream_t s);

}  // namespace esdg
