// Host-side launch wrappers, one explicit instantiation per degree N (the
// esdg_kernels_nK.cu translation units compile in parallel).
#pragma once

#include <cuda_runtime.h>

#include "esdg_kernels.cuh"
#include "esdg_ensemble.cuh"

namespace esdg {

// Launch geometry of the persistent warp-per-element kernels (k_stage for the
// FP64 right-hand side, k_project for both precisions): CTAs of 8 warps, as
// many CTAs per SM as fit.
struct LaunchGeom {
    int block = 256;
    int grid = 0;
    size_t smem = 0;
};

template <int N, typename real>
cudaError_t stage_geometry(int num_sms, LaunchGeom& lg);
template <int N, typename real>
cudaError_t project_geometry(int num_sms, LaunchGeom& lg);
template <int N, typename real>
cudaError_t launch_project(const StageParams<real>& p, const LaunchGeom& lg, cudaStream_t s);
template <int N, typename real>
cudaError_t launch_stage(const StageParams<real>& p, int mode, const LaunchGeom& lg, cudaStream_t s);
// FP32 batched stage kernel (esdg_stage2.cuh): one CTA of 12 warps per SM.
template <int N>
cudaError_t stage2_geometry(int num_sms, LaunchGeom& lg);
template <int N>
cudaError_t launch_stage2(const StageParams<float>& p, const float* ops2, int Kpad, int mode, const LaunchGeom& lg,
                          cudaStream_t s);
template <int N>
cudaError_t launch_entropy(int K, double g, const double* u, const double* rhs, const double* Vq, const double* wJq,
                           const double* bq, double* partial, int nparts, double* out, cudaStream_t s);
// DG-SBP kernels (esdg_sbp.cuh), degree N = 1..5, FP64 and FP32.
template <int N, typename real>
cudaError_t sbp_geometry(int num_sms, LaunchGeom& lg);
template <int N, typename real>
cudaError_t launch_sbp(const StageParams<real>& p, int mode, const LaunchGeom& lg, cudaStream_t s);
// FP32 batched DG-SBP stage kernel (esdg_sbp2.cuh), modes 0 and 1.
template <int N>
cudaError_t sbp2_geometry(int num_sms, LaunchGeom& lg);
template <int N>
cudaError_t launch_sbp2(const StageParams<float>& p, const float* ops2, int Kpad, int mode, const LaunchGeom& lg,
                        cudaStream_t s);
int sbp2_ops_floats(int N);
cudaError_t launch_entropy_nodal(int K, int Nq, double g, const double* u, const double* rhs, const double* wJq,
                                 const double* bq, double* partial, int nparts, double* out, cudaStream_t s);
// FP64 L2 error against given values at the volume points (esdg_diag.cu):
// Vq [Nq][Np] for a modal state, NULL for a nodal one (Np = Nq).
cudaError_t launch_l2_error(int K, int Nq, int Np, const double* u, const double* Vq, const double* wJq,
                            const double* exact, double* partial, int nparts, double* out, cudaStream_t s);

}  // namespace esdg
