// DG-SBP kernels with an FP32 right-hand side (FP64 state and RK update): the
// generic kernel (record preparation) and the batched stage kernel.
#define ESDG_SBP_REAL float
#include "esdg_sbp_impl.cuh"
#include "esdg_sbp2.cuh"

namespace esdg {

template <int N>
cudaError_t sbp2_geometry(int num_sms, LaunchGeom& lg) {
    lg.block = 32 * S2<N>::WARPS;
    lg.smem = S2<N>::bytes();
    cudaError_t err;
    err = cudaFuncSetAttribute(k_sbp2<N, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(k_sbp2<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lg.smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sbp2<N, 1>, lg.block, lg.smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    lg.grid = per_sm * num_sms;
    return cudaSuccess;
}

template <int N>
cudaError_t launch_sbp2(const StageParams<float>& p, const float* ops2, int Kpad, int mode, const LaunchGeom& lg,
                        cudaStream_t s) {
    const int batches = Kpad / S2<N>::EPW;
    const int need = (batches + S2<N>::WARPS - 1) / S2<N>::WARPS;
    const int grid = need < lg.grid ? need : lg.grid;
    if (mode == 0)
        k_sbp2<N, 0><<<grid, lg.block, lg.smem, s>>>(p, ops2, Kpad);
    else
        k_sbp2<N, 1><<<grid, lg.block, lg.smem, s>>>(p, ops2, Kpad);
    return cudaGetLastError();
}

int sbp2_ops_floats(int N) {
    switch (N) {
        case 1: return S2<1>::o_end;
        case 2: return S2<2>::o_end;
        case 3: return S2<3>::o_end;
        case 4: return S2<4>::o_end;
        case 5: return S2<5>::o_end;
    }
    return 0;
}

#define ESDG_SBP2_INST(n)                                                                                        \
    template cudaError_t sbp2_geometry<n>(int, LaunchGeom&);                                                    \
    template cudaError_t launch_sbp2<n>(const StageParams<float>&, const float*, int, int, const LaunchGeom&, \
                                        cudaStream_t);
ESDG_SBP2_INST(1)
ESDG_SBP2_INST(2)
ESDG_SBP2_INST(3)
ESDG_SBP2_INST(4)
ESDG_SBP2_INST(5)
#undef ESDG_SBP2_INST

}  // namespace esdg
