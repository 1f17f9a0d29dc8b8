// Volume-kernel cost comparison of Sec. 5.4: the traditional DG volume term
// (matrix-vector products Q^x f^x(u) + Q^y f^y(u), one flux evaluation per
// node) against the entropy-stable flux-differencing term
// (Q^x o F^x) 1 + (Q^y o F^y) 1 (one two-point flux evaluation per matrix
// entry), with dense n x n operators (random entries in the comparison) and
// the shallow-water fluxes of eq. (SWE) and eqs. (SWE_flux1/2).
//
// GPU: one CTA per EV elements, one thread per row j (blockDim = n rounded up
// to a warp); the operators stream through shared memory in column tiles of
// TJ, stored transposed so a column tile is read conflict-free; the node data
// of the CTA's elements sit in shared memory.  Both kernels share this
// structure, so their ratio measures the cost of the two-point fluxes.
//
// The ESDG sum uses sums instead of averages: with s_a = a_j + a_k,
//   F^x = (s_hu / 2, s_hu s_u / 4 + p, s_hu s_v / 4),
//   F^y = (s_hv / 2, s_hv s_u / 4, s_hv s_v / 4 + p),
//   p = g {h}^2 - g {h^2} / 2 = g (s_h^2 - s_h2) / 4,
// so with T = Q^x s_hu + Q^y s_hv the row sums are (sum T / 2,
// sum (s_u T + 4 Q^x p) / 4, sum (s_v T + 4 Q^y p) / 4).
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "esdg.h"

namespace {

constexpr int EV = 4;    // elements per CTA
constexpr int TJ = 32;   // operator columns per shared-memory tile
constexpr int NMAX = 256;

template <typename real>
__global__ void __launch_bounds__(NMAX) k_volume(int kind, int n, int K, real g, const real* __restrict__ Qx,
                                                  const real* __restrict__ Qy, const real* __restrict__ u,
                                                  real* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* qx = reinterpret_cast<real*>(smem_raw);   // [TJ][n]: qx[kk * n + j] = Qx[j][k0 + kk]
    real* qy = qx + TJ * n;
    real* nd = qy + TJ * n;                         // [EV][6][n] node data
    const int e0 = blockIdx.x * EV;
    const int j = threadIdx.x;
    // node data: DG -> f^x (3), f^y (3); ESDG -> h, hu, hv, u, v, h^2
    for (int idx = threadIdx.x; idx < EV * n; idx += blockDim.x) {
        const int e = idx / n, k = idx - e * n;
        real h = 1, hu = 0, hv = 0;
        if (e0 + e < K) {
            h = u[((size_t)0 * K + e0 + e) * n + k];
            hu = u[((size_t)1 * K + e0 + e) * n + k];
            hv = u[((size_t)2 * K + e0 + e) * n + k];
        }
        const real uu = hu / h, vv = hv / h;
        real* d = nd + (size_t)e * 6 * n + k;
        if (kind == ESDG_VOLUME_DG) {
            const real p = real(0.5) * g * h * h;
            d[0 * n] = hu;
            d[1 * n] = hu * uu + p;
            d[2 * n] = hu * vv;
            d[3 * n] = hv;
            d[4 * n] = hv * uu;
            d[5 * n] = hv * vv + p;
        } else {
            d[0 * n] = h;
            d[1 * n] = hu;
            d[2 * n] = hv;
            d[3 * n] = uu;
            d[4 * n] = vv;
            d[5 * n] = h * h;
        }
    }
    real a0[EV], a1[EV], a2[EV];
    real rh[EV], rhu[EV], rhv[EV], ru[EV], rv[EV], rh2[EV];
#pragma unroll
    for (int e = 0; e < EV; ++e) a0[e] = a1[e] = a2[e] = 0;
    __syncthreads();
    if (kind == ESDG_VOLUME_ESDG && j < n) {
#pragma unroll
        for (int e = 0; e < EV; ++e) {
            const real* d = nd + (size_t)e * 6 * n + j;
            rh[e] = d[0];
            rhu[e] = d[n];
            rhv[e] = d[2 * n];
            ru[e] = d[3 * n];
            rv[e] = d[4 * n];
            rh2[e] = d[5 * n];
        }
    }
    const real g4 = g;  // p4 = 4 p = g (s_h^2 - s_h2)
    for (int k0 = 0; k0 < n; k0 += TJ) {
        const int tk = n - k0 < TJ ? n - k0 : TJ;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * tk; idx += blockDim.x) {
            const int jj = idx / tk, kk = idx - jj * tk;  // coalesced along kk (a row segment of Q)
            qx[kk * n + jj] = Qx[(size_t)jj * n + k0 + kk];
            qy[kk * n + jj] = Qy[(size_t)jj * n + k0 + kk];
        }
        __syncthreads();
        if (j >= n) continue;
        if (kind == ESDG_VOLUME_DG) {
            for (int kk = 0; kk < tk; ++kk) {
                const real cx = qx[kk * n + j], cy = qy[kk * n + j];
#pragma unroll
                for (int e = 0; e < EV; ++e) {
                    const real* d = nd + (size_t)e * 6 * n + k0 + kk;
                    a0[e] += cx * d[0] + cy * d[3 * n];
                    a1[e] += cx * d[n] + cy * d[4 * n];
                    a2[e] += cx * d[2 * n] + cy * d[5 * n];
                }
            }
        } else {
            for (int kk = 0; kk < tk; ++kk) {
                const real cx = qx[kk * n + j], cy = qy[kk * n + j];
#pragma unroll
                for (int e = 0; e < EV; ++e) {
                    const real* d = nd + (size_t)e * 6 * n + k0 + kk;
                    const real sh = rh[e] + d[0], shu = rhu[e] + d[n], shv = rhv[e] + d[2 * n];
                    const real su = ru[e] + d[3 * n], sv = rv[e] + d[4 * n], sh2 = rh2[e] + d[5 * n];
                    const real p4 = g4 * (sh * sh - sh2);
                    const real T = cx * shu + cy * shv;
                    a0[e] += T;
                    a1[e] += su * T + cx * p4;
                    a2[e] += sv * T + cy * p4;
                }
            }
        }
    }
    if (j >= n) return;
    const real s0 = kind == ESDG_VOLUME_ESDG ? real(0.5) : real(1);
    const real s1 = kind == ESDG_VOLUME_ESDG ? real(0.25) : real(1);
#pragma unroll
    for (int e = 0; e < EV; ++e) {
        if (e0 + e >= K) break;
        out[((size_t)0 * K + e0 + e) * n + j] = s0 * a0[e];
        out[((size_t)1 * K + e0 + e) * n + j] = s1 * a1[e];
        out[((size_t)2 * K + e0 + e) * n + j] = s1 * a2[e];
    }
}

template <typename real>
int launch(int kind, int n, int K, double g, const void* Qx, const void* Qy, const void* u, void* out,
           cudaStream_t s) {
    const int block = (n + 31) / 32 * 32;
    const size_t smem = sizeof(real) * (size_t(2) * TJ * n + size_t(EV) * 6 * n);
    cudaError_t e = cudaFuncSetAttribute(k_volume<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return ESDG_ECUDA;
    k_volume<real><<<(K + EV - 1) / EV, block, smem, s>>>(kind, n, K, (real)g, static_cast<const real*>(Qx),
                                                         static_cast<const real*>(Qy), static_cast<const real*>(u),
                                                         static_cast<real*>(out));
    return cudaGetLastError() == cudaSuccess ? ESDG_OK : ESDG_ECUDA;
}

// The same two volume terms on the host, one thread, plain loops (the CPU side
// of the comparison).
template <typename real>
void host_volume(int kind, int n, int K, real g, const real* Qx, const real* Qy, const real* u, real* out) {
    std::vector<real> d(6 * size_t(n));
    for (int e = 0; e < K; ++e) {
        for (int k = 0; k < n; ++k) {
            const real h = u[((size_t)0 * K + e) * n + k], hu = u[((size_t)1 * K + e) * n + k];
            const real hv = u[((size_t)2 * K + e) * n + k];
            const real uu = hu / h, vv = hv / h;
            if (kind == ESDG_VOLUME_DG) {
                const real p = real(0.5) * g * h * h;
                d[0 * n + k] = hu;
                d[1 * n + k] = hu * uu + p;
                d[2 * n + k] = hu * vv;
                d[3 * n + k] = hv;
                d[4 * n + k] = hv * uu;
                d[5 * n + k] = hv * vv + p;
            } else {
                d[0 * n + k] = h;
                d[1 * n + k] = hu;
                d[2 * n + k] = hv;
                d[3 * n + k] = uu;
                d[4 * n + k] = vv;
                d[5 * n + k] = h * h;
            }
        }
        for (int j = 0; j < n; ++j) {
            real a0 = 0, a1 = 0, a2 = 0;
            const real* qx = Qx + (size_t)j * n;
            const real* qy = Qy + (size_t)j * n;
            if (kind == ESDG_VOLUME_DG) {
                for (int k = 0; k < n; ++k) {
                    a0 += qx[k] * d[k] + qy[k] * d[3 * n + k];
                    a1 += qx[k] * d[n + k] + qy[k] * d[4 * n + k];
                    a2 += qx[k] * d[2 * n + k] + qy[k] * d[5 * n + k];
                }
                out[((size_t)0 * K + e) * n + j] = a0;
                out[((size_t)1 * K + e) * n + j] = a1;
                out[((size_t)2 * K + e) * n + j] = a2;
            } else {
                const real rh = d[j], rhu = d[n + j], rhv = d[2 * n + j], ru = d[3 * n + j], rv = d[4 * n + j];
                const real rh2 = d[5 * n + j];
                for (int k = 0; k < n; ++k) {
                    const real sh = rh + d[k], shu = rhu + d[n + k], shv = rhv + d[2 * n + k];
                    const real su = ru + d[3 * n + k], sv = rv + d[4 * n + k], sh2 = rh2 + d[5 * n + k];
                    const real p4 = g * (sh * sh - sh2);
                    const real T = qx[k] * shu + qy[k] * shv;
                    a0 += T;
                    a1 += su * T + qx[k] * p4;
                    a2 += sv * T + qy[k] * p4;
                }
                out[((size_t)0 * K + e) * n + j] = real(0.5) * a0;
                out[((size_t)1 * K + e) * n + j] = real(0.25) * a1;
                out[((size_t)2 * K + e) * n + j] = real(0.25) * a2;
            }
        }
    }
}

int check_args(int kind, int precision, int n, int K, const void* Qx, const void* Qy, const void* u,
               const void* out) {
    if (kind != ESDG_VOLUME_DG && kind != ESDG_VOLUME_ESDG) return ESDG_EINVAL;
    if (precision != ESDG_FP32 && precision != ESDG_FP64) return ESDG_EINVAL;
    if (n < 1 || n > NMAX || K < 1) return ESDG_EINVAL;
    if (!Qx || !Qy || !u || !out) return ESDG_EINVAL;
    return ESDG_OK;
}

}  // namespace

extern "C" {

int esdg_volume_kernel(int kind, int precision, int n, int K, double g, const void* Qx, const void* Qy,
                       const void* u, void* out, void* stream) {
    int rc = check_args(kind, precision, n, K, Qx, Qy, u, out);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return precision == ESDG_FP32 ? launch<float>(kind, n, K, g, Qx, Qy, u, out, s)
                                  : launch<double>(kind, n, K, g, Qx, Qy, u, out, s);
}

int esdg_volume_kernel_host(int kind, int precision, int n, int K, double g, const void* Qx, const void* Qy,
                            const void* u, void* out) {
    int rc = check_args(kind, precision, n, K, Qx, Qy, u, out);
    if (rc) return rc;
    if (precision == ESDG_FP32)
        host_volume<float>(kind, n, K, (float)g, static_cast<const float*>(Qx), static_cast<const float*>(Qy),
                           static_cast<const float*>(u), static_cast<float*>(out));
    else
        host_volume<double>(kind, n, K, g, static_cast<const double*>(Qx), static_cast<const double*>(Qy),
                            static_cast<const double*>(u), static_cast<double*>(out));
    return ESDG_OK;
}

}  // extern "C"
