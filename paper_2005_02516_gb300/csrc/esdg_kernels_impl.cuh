// Definitions of the launch wrappers for one degree N (ESDG_N).
#include "esdg_launch.hpp"

namespace esdg {

// the RK-stage kernel of degree N (the three-block form where it applies)
template <int N, typename real>
static auto stage_kernel1() {
    if constexpr (k_stage_three_blocks<N, 1>())
        return &k_stage<N, real, 1, 3>;
    else
        return &k_stage<N, real, 1>;
}

template <int N, typename real>
cudaError_t stage_geometry(int num_sms, LaunchGeom& lg) {
    lg.block = 256;
    lg.smem = Smem<N, real>::bytes(lg.block / 32);
    cudaError_t err;
    err = cudaFuncSetAttribute(k_stage<N, real, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    auto* k1 = stage_kernel1<N, real>();
    err = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1, lg.block, lg.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    lg.grid = per_sm * num_sms;
    return cudaSuccess;
}

template <int N, typename real>
cudaError_t project_geometry(int num_sms, LaunchGeom& lg) {
    lg.block = 256;
    lg.smem = Smem<N, real>::bytes(lg.block / 32);
    cudaError_t err =
        cudaFuncSetAttribute(k_project<N, real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project<N, real>, lg.block, lg.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    lg.grid = per_sm * num_sms;
    return cudaSuccess;
}

template <int N, typename real>
cudaError_t launch_project(const StageParams<real>& p, const LaunchGeom& lg, cudaStream_t s) {
    int need = (p.K + lg.block / 32 - 1) / (lg.block / 32);
    int grid = need < lg.grid ? need : lg.grid;
    k_project<N, real><<<grid, lg.block, lg.smem, s>>>(p);
    return cudaGetLastError();
}

template <int N, typename real>
cudaError_t launch_stage(const StageParams<real>& p, int mode, const LaunchGeom& lg, cudaStream_t s) {
    int need = (p.K + lg.block / 32 - 1) / (lg.block / 32);
    int grid = need < lg.grid ? need : lg.grid;
    if (mode == 0)
        k_stage<N, real, 0><<<grid, lg.block, lg.smem, s>>>(p);
    else
        stage_kernel1<N, real>()<<<grid, lg.block, lg.smem, s>>>(p);
    return cudaGetLastError();
}

template <int N>
cudaError_t stage2_geometry(int num_sms, LaunchGeom& lg) {
    lg.block = 32 * C2<N>::WARPS;
    lg.smem = C2<N>::bytes();
    cudaError_t err;
    err = cudaFuncSetAttribute(k_stage2<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_stage2<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_stage2<N, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage2<N, 1>, lg.block, lg.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    lg.grid = per_sm * num_sms;
    return cudaSuccess;
}

template <int N>
cudaError_t launch_stage2(const StageParams<float>& p, const float* ops2, int Kpad, int mode, const LaunchGeom& lg,
                          cudaStream_t s) {
    const int batches = Kpad / C2<N>::EPW;
    const int need = (batches + C2<N>::WARPS - 1) / C2<N>::WARPS;
    const int grid = need < lg.grid ? need : lg.grid;
    if (mode == 0)
        k_stage2<N, 0><<<grid, lg.block, lg.smem, s>>>(p, ops2, Kpad);
    else if (mode == 1)
        k_stage2<N, 1><<<grid, lg.block, lg.smem, s>>>(p, ops2, Kpad);
    else
        k_stage2<N, 2><<<grid, lg.block, lg.smem, s>>>(p, ops2, Kpad);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_entropy(int K, double g, const double* u, const double* rhs, const double* Vq, const double* wJq,
                           const double* bq, double* partial, int nparts, double* out, cudaStream_t s) {
    k_entropy<N><<<nparts, 256, 0, s>>>(K, g, u, rhs, Vq, wJq, bq, partial);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_entropy_finalize<<<1, 32, 0, s>>>(nparts, partial, out);
    return cudaGetLastError();
}

template cudaError_t stage2_geometry<ESDG_N>(int, LaunchGeom&);
template cudaError_t launch_stage2<ESDG_N>(const StageParams<float>&, const float*, int, int, const LaunchGeom&,
                                          cudaStream_t);
#ifndef ESDG_STAGE2_ONLY  // the tensor-core forms (ESDG_N >= 32) have the FP32 stage kernel only
template cudaError_t stage_geometry<ESDG_N, double>(int, LaunchGeom&);
template cudaError_t project_geometry<ESDG_N, double>(int, LaunchGeom&);
template cudaError_t launch_project<ESDG_N, double>(const StageParams<double>&, const LaunchGeom&, cudaStream_t);
template cudaError_t launch_stage<ESDG_N, double>(const StageParams<double>&, int, const LaunchGeom&, cudaStream_t);
template cudaError_t launch_entropy<ESDG_N>(int, double, const double*, const double*, const double*, const double*,
                                            const double*, double*, int, double*, cudaStream_t);
#endif

}  // namespace esdg
