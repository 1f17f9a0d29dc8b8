// Ensemble kernel: one LSRK45 stage of several independent ESDG problems of
// mixed degree and size in one persistent launch (see esdg_stage2.cuh for the
// per-batch arithmetic and EnsembleMember for the tile table).  Included once
// per volume rule, with ESDG_RULE defined (esdg_ensemble.cu: collapsed,
// esdg_ensemble_s.cu: symmetric).
#include "esdg_ensemble.cuh"

namespace esdg {

// One batch of a member of degree NR: a call, not inlined, so that each
// degree's body is allocated registers on its own.
template <int NR>
__device__ __noinline__ bool ensemble_batch(const StageParams<float>& p, const float* __restrict__ ut_in,
                                            float* __restrict__ ut_out, double rkA, double rkB,
                                            const float* __restrict__ ops, float* ws, uint64_t* bar,
                                            uint32_t& parity, int e0, int lane) {
    return stage2_batch<NR, 1>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane);
}

// One LSRK45 stage for every member.  ops_off[N]: float offset of degree N's
// operators in shared memory (-1 if no member has that degree); slab: floats
// per warp region (the largest over the degrees present).
template <int NMAX, int RULE>
__global__ void __launch_bounds__(ensemble_max_warps(NMAX) * 32, 1)
k_stage2_ensemble(const EnsembleMember* __restrict__ mem, int nmem, int total_batches, int which, double rkA,
                  double rkB, int4 ops_lo, int ops_hi, int ops_end, int slab) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    const int nwarps = blockDim.x >> 5;
    int* tile = reinterpret_cast<int*>(sm + ops_end + nwarps * slab);          // [nmem + 1] batch starts
    uint64_t* bars = reinterpret_cast<uint64_t*>(tile + ((nmem + 1 + 3) & ~3));
    // operators of every degree present (from the first member of that degree)
    for (int n = 1; n <= 5; ++n) {
        const int off = n == 1 ? ops_lo.x : n == 2 ? ops_lo.y : n == 3 ? ops_lo.z : n == 4 ? ops_lo.w : ops_hi;
        if (off < 0) continue;
        int first = 0;
        while (first < nmem && mem[first].N != n) ++first;
        constexpr int R8 = 8 * RULE;
        const int cnt = n == 1 ? C2<1 + R8>::o_end : n == 2 ? C2<2 + R8>::o_end : n == 3 ? C2<3 + R8>::o_end
                        : n == 4 ? C2<4 + R8>::o_end : C2<5 + R8>::o_end;
        const float4* src = reinterpret_cast<const float4*>(mem[first].ops2);
        float4* dst = reinterpret_cast<float4*>(sm + off);
        for (int i = threadIdx.x; i < cnt / 4; i += blockDim.x) dst[i] = src[i];
    }
    for (int i = threadIdx.x; i < nmem; i += blockDim.x) tile[i] = mem[i].batch_begin;
    if (threadIdx.x == 0) tile[nmem] = total_batches;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) mbar_init(&bars[warp], 1);
    fence_mbar_init();
    __syncthreads();
    uint64_t* bar = &bars[warp];
    float* ws = sm + ops_end + warp * slab;
    // the current member's parameters, copied into this warp's slot of shared
    // memory when the member changes: read from there they take no registers
    // through the batch (read from the member table in global memory they
    // would be loaded early and held)
    StageParams<float>* pw = reinterpret_cast<StageParams<float>*>(bars + nwarps) + warp;
    int cur = -1;
    uint32_t parity = 0;
    for (int gb = blockIdx.x * nwarps + warp; gb < total_batches; gb += gridDim.x * nwarps) {
        int lo = 0, hi = nmem - 1;  // the member whose batch range holds gb
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tile[mid] <= gb) lo = mid; else hi = mid - 1;
        }
        const EnsembleMember& M = mem[lo];
        if (lo != cur) {
            __syncwarp();
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&M.p);
            uint32_t* dst = reinterpret_cast<uint32_t*>(pw);
            for (int i = lane; i < (int)(sizeof(StageParams<float>) / 4); i += 32) dst[i] = src[i];
            __syncwarp();
            cur = lo;
        }
        const StageParams<float>& p = *pw;
        const float* ut_in = M.ut[which];
        float* ut_out = M.ut[which ^ 1];
        const int e0 = (gb - tile[lo]) * 4;
        const int n = M.N;
        const float* ops = sm + (n == 1 ? ops_lo.x : n == 2 ? ops_lo.y : n == 3 ? ops_lo.z : n == 4 ? ops_lo.w : ops_hi);
        bool ok = true;
        switch (n) {
            case 1: ok = ensemble_batch<1 + 8 * RULE>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane); break;
            case 2: ok = ensemble_batch<2 + 8 * RULE>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane); break;
            case 3: ok = ensemble_batch<3 + 8 * RULE>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane); break;
            case 4: ok = ensemble_batch<4 + 8 * RULE>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane); break;
            default:
                if (NMAX >= 5) ok = ensemble_batch<5 + 8 * RULE>(p, ut_in, ut_out, rkA, rkB, ops, ws, bar, parity, e0, lane);
                break;
        }
        if (!ok) return;
    }
}

template <int RULE>
cudaError_t ensemble_smem_attr(int nmax, size_t smem) {
    if (nmax <= 4)
        return cudaFuncSetAttribute(k_stage2_ensemble<4, RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    return cudaFuncSetAttribute(k_stage2_ensemble<5, RULE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int RULE>
cudaError_t launch_ensemble(int nmax, int grid, int block, size_t smem, cudaStream_t s, const EnsembleMember* mem,
                            int nmem, int total_batches, int which, double rkA, double rkB, int4 ops_lo, int ops_hi,
                            int ops_end, int slab) {
    if (nmax <= 4)
        k_stage2_ensemble<4, RULE><<<grid, block, smem, s>>>(mem, nmem, total_batches, which, rkA, rkB, ops_lo, ops_hi,
                                                        ops_end, slab);
    else
        k_stage2_ensemble<5, RULE><<<grid, block, smem, s>>>(mem, nmem, total_batches, which, rkA, rkB, ops_lo, ops_hi,
                                                        ops_end, slab);
    return cudaGetLastError();
}

template cudaError_t ensemble_smem_attr<ESDG_RULE>(int, size_t);
template cudaError_t launch_ensemble<ESDG_RULE>(int, int, int, size_t, cudaStream_t, const EnsembleMember*, int, int,
                                                int, double, double, int4, int, int, int);

}  // namespace esdg
