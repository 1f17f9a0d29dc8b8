// Launch wrappers and instantiations of the DG-SBP kernels for one
// arithmetic type (ESDG_SBP_REAL), degrees 1..5.
#include "esdg_launch.hpp"
#include "esdg_sbp.cuh"

namespace esdg {

template <int N, typename real>
cudaError_t sbp_geometry(int num_sms, LaunchGeom& lg) {
    lg.block = 256;
    lg.smem = SbpSmem<N, real>::bytes(lg.block / 32);
    cudaError_t err;
    err = cudaFuncSetAttribute(k_sbp<N, real, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_sbp<N, real, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_sbp<N, real, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbp<N, real, 1>, lg.block, lg.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    lg.grid = per_sm * num_sms;
    return cudaSuccess;
}

template <int N, typename real>
cudaError_t launch_sbp(const StageParams<real>& p, int mode, const LaunchGeom& lg, cudaStream_t s) {
    const int need = (p.K + lg.block / 32 - 1) / (lg.block / 32);
    const int grid = need < lg.grid ? need : lg.grid;
    if (mode == 0)
        k_sbp<N, real, 0><<<grid, lg.block, lg.smem, s>>>(p);
    else if (mode == 1)
        k_sbp<N, real, 1><<<grid, lg.block, lg.smem, s>>>(p);
    else
        k_sbp<N, real, 2><<<grid, lg.block, lg.smem, s>>>(p);
    return cudaGetLastError();
}

#define ESDG_SBP_INST(n)                                                                                  \
    template cudaError_t sbp_geometry<n, ESDG_SBP_REAL>(int, LaunchGeom&);                               \
    template cudaError_t launch_sbp<n, ESDG_SBP_REAL>(const StageParams<ESDG_SBP_REAL>&, int, const LaunchGeom&, \
                                                      cudaStream_t);
ESDG_SBP_INST(1)
ESDG_SBP_INST(2)
ESDG_SBP_INST(3)
ESDG_SBP_INST(4)
ESDG_SBP_INST(5)
#undef ESDG_SBP_INST

}  // namespace esdg
