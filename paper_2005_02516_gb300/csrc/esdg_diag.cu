// FP64 L2 error of the state against values given at the volume points (the
// error measure of the convergence study in Sec. 4.1, evaluated with the
// element's own volume rule): per field f,
//   err_f^2 = sum_k sum_q w_q J_q^k (u_q[f] - exact[f][k][q])^2,
// u_q = V_q u_h for a modal state, the nodal values for a DG-SBP state.
#include <cuda_runtime.h>

#include "esdg_kernels.cuh"
#include "esdg_launch.hpp"

namespace esdg {

__global__ void __launch_bounds__(256) k_l2_error(int K, int Nq, int Np, const double* __restrict__ u,
                                                  const double* __restrict__ Vq, const double* __restrict__ wJq,
                                                  const double* __restrict__ exact, double* __restrict__ partial) {
    double s[3] = {0.0, 0.0, 0.0};
    const size_t total = (size_t)K * Nq;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx / Nq), q = (int)(idx - (size_t)e * Nq);
        const double w = wJq[idx];
        for (int c = 0; c < 3; ++c) {
            double uq;
            if (Vq) {
                uq = 0.0;
                const double* ue = u + ((size_t)c * K + e) * Np;
                for (int n = 0; n < Np; ++n) uq += Vq[q * Np + n] * ue[n];
            } else {
                uq = u[(size_t)c * total + idx];
            }
            const double d = uq - exact[(size_t)c * total + idx];
            s[c] += w * d * d;
        }
    }
    __shared__ double red[3][256];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) partial[blockIdx.x * 3 + c] = red[c][0];
}

cudaError_t launch_l2_error(int K, int Nq, int Np, const double* u, const double* Vq, const double* wJq,
                            const double* exact, double* partial, int nparts, double* out, cudaStream_t s) {
    k_l2_error<<<nparts, 256, 0, s>>>(K, Nq, Np, u, Vq, wJq, exact, partial);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_entropy_finalize<<<1, 32, 0, s>>>(nparts, partial, out);
    return cudaGetLastError();
}

}  // namespace esdg
