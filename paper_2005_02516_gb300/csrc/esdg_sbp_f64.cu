// DG-SBP kernels in FP64, and the FP64 diagnostics of nodal states.
#define ESDG_SBP_REAL double
#include "esdg_sbp_impl.cuh"

namespace esdg {

__global__ void __launch_bounds__(256) k_entropy_nodal(int K, int Nq, double g, const double* __restrict__ u,
                                                       const double* __restrict__ rhs,
                                                       const double* __restrict__ wJq,
                                                       const double* __restrict__ bq, double* __restrict__ partial) {
    double s_ent = 0, s_mass = 0, s_rate = 0;
    const size_t total = (size_t)K * Nq;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const double h = u[idx], hu = u[total + idx], hv = u[2 * total + idx];
        const double w = wJq[idx], b = bq[idx];
        const double uu = hu / h, vv = hv / h;
        s_ent += w * (0.5 * (hu * uu + hv * vv) + 0.5 * g * h * h + g * h * b);
        s_mass += w * h;
        if (rhs)
            s_rate += w * ((g * (h + b) - 0.5 * (uu * uu + vv * vv)) * rhs[idx] + uu * rhs[total + idx] +
                           vv * rhs[2 * total + idx]);
    }
    __shared__ double red[3][256];
    red[0][threadIdx.x] = s_ent;
    red[1][threadIdx.x] = s_mass;
    red[2][threadIdx.x] = s_rate;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) partial[blockIdx.x * 3 + c] = red[c][0];
}

cudaError_t launch_entropy_nodal(int K, int Nq, double g, const double* u, const double* rhs, const double* wJq,
                                 const double* bq, double* partial, int nparts, double* out, cudaStream_t s) {
    k_entropy_nodal<<<nparts, 256, 0, s>>>(K, Nq, g, u, rhs, wJq, bq, partial);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_entropy_finalize<<<1, 32, 0, s>>>(nparts, partial, out);
    return cudaGetLastError();
}

}  // namespace esdg
