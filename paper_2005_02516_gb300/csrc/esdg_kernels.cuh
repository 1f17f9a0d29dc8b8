// CUDA kernels of the ESDG shallow-water right-hand side and LSRK45 stage
// (Wu, Kubatko, Chan, arXiv 2005.02516).  Written for sm_103a.
//
// Per RK stage one fused kernel does, per element (a warp per element):
//   volume flux differencing with the entropy-conservative SWE flux
//   (eqs. (SWE_flux1/2)) and its well-balanced bathymetry term, on the skew
//   hybridized operator of Sec. 5.2 (Q_skew = Q_h - Q_h^T, whose lower-right
//   block is zero and skipped), with the curved metric average of Sec. 2.7;
//   the interface flux f_S(u~+, u~) with Lax-Friedrichs (Sec. 2.8);
//   the lift V_h^T and the stored inverse curved mass matrix (Sec. 2.7, 5.1);
//   the LSRK45 stage update in FP64 (Sec. 4);
//   and the entropy projection (Sec. 2.6) of the updated state, written for
//   the next stage (its face values are what neighbours read).
//
// Algebra used by the volume loop.  With sums over the pair (l, m)
//   HU = hu_l + hu_m, HV = hv_l + hv_m, U = u_l + u_m, V = v_l + v_m,
// and the metric average folded into the operator entries
//   Qx = 1/4 Qskew^x[l,m] = qr (rx_l + rx_m) + qs (sx_l + sx_m), (metrics / 8)
// the row-l contribution of Qskew^x o F^x + Qskew^y o F^y is
//   h  : 2 (Qx HU + Qy HV)
//   hu : U (Qx HU + Qy HV) + Qx * 2 g h_l H_m
//   hv : V (Qx HU + Qy HV) + Qy * 2 g h_l H_m
// where the pressure g{h}^2 - g{h^2}/2 = g h_l h_m / 2 and the source
// -g h~ (1/2 Qskew b) combine into g/2 h_l (h_m + b_m) = g/2 h_l H_m.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace esdg {

// Points of the fully symmetric volume rule exact to degree 2N.
constexpr int symmetric_points(int N) { return N == 1 ? 3 : N == 2 ? 6 : N == 3 ? 12 : N == 4 ? 16 : 25; }

// Template parameter NR = N + 8 * rule + 16 * wadg: the degree N (1..5), the
// volume rule (0: collapsed (N+1)^2 points, 1: symmetric, exact to 2N) and the
// inverse mass matrix (0: the stored (M_h^k)^{-1} of Sec. 2.7; 1: the
// weight-adjusted inverse M^{-1} M_{1/J} M^{-1} = Vq^T W diag(1/J) Vq applied
// on the fly, the alternative Sec. 2.8 names; M = I for these rules), plus
// 32 * tc for the FP32 kernel whose dense contractions run on the tensor cores.
template <int NR>
struct Dims {
    static constexpr int N = NR & 7;
    static constexpr int rule = (NR >> 3) & 1;
    static constexpr int wadg = (NR >> 4) & 1;
    static constexpr int tc = (NR >> 5) & 1;    // dense contractions on the tensor cores (FP32 kernel)
    static constexpr int Np = (N + 1) * (N + 2) / 2;
    static constexpr int Nq = rule ? symmetric_points(N) : (N + 1) * (N + 1);
    static constexpr int Nfp = N + 1;
    static constexpr int Nfq = 3 * (N + 1);
    static constexpr int Nh = Nq + Nfq;
    static constexpr int NpP = Np * (Np + 1) / 2;
};

// The FP64 kernel's unique-pair schedule (rules with Nq <= 16 and Nh <= 32):
// volume-volume pairs along the diagonals (j, j + d mod V), d = 1..SVV, the
// two half-warps taking d <= SVV0 and d > SVV0; volume-face pairs along
// (j, V + (j + t) mod L), t < L, split the same way: NSTEP steps in all.
template <int NR>
struct PairSched {
    typedef Dims<NR> D;
    static constexpr bool SPLIT = D::Nq <= 16 && D::Nh <= 32;
    static constexpr int V = D::Nq, F = D::Nfq, L = V > F ? V : F;
    static constexpr int SVV = V / 2, SVV0 = (SVV + 1) / 2, SVF0 = (L + 1) / 2;
    static constexpr int NSTEP = SVV0 + SVF0;
};

// status bits written by the device
constexpr int STATUS_NONPOSITIVE = 1;
constexpr int STATUS_NONFINITE = 2;

template <typename real>
struct StageParams {
    int K;
    real g;
    int lf;
    // reference operators (global, staged into shared memory)
    const real* QsT;   // [Nh(m)][Nh(l)][2]: (Qskew^r[l][m], Qskew^s[l][m])
    const real* Vq;    // [Nq][Np]
    const real* VqT;   // [Np][Nq]
    const real* Vh;    // [Nh][Np]
    const real* VhT;   // [Np][Nh]
    const real* wf;    // [Nfq]
    const real* nrs;   // [Nfq][2] scaled reference normals
    const real* wq;    // [Nq]     volume weights (weight-adjusted inverse: w_q / J_q = w_q^2 / (w_q J_q))
    const real* iwJ;   // [K][Nq]  DG-SBP FP64: 1 / (w_q J_q), the inverse of the diagonal mass (else null)
    const int* fmap;   // [Nfq]    DG-SBP: the volume node of each face node (the selection I_f)
    // per element
    const real* geo;   // [K][Nh][4] rxJ sxJ ryJ syJ
    const real* wJq;   // [K][Nq]   w_q J_q
    const real* minv;  // [K][mstride] packed (M_h^k)^{-1} (stored inverse only)
    int mstride;       // element stride of minv (NpP rounded up to a multiple of 4)
    const real* bh;    // [K][Nh]   bathymetry at hybrid nodes
    const int* nbr;    // [K][3]    4 * neighbour element + neighbour face (4 e + 3: wall)
    int walls;         // reflective walls present (Sec. 2.9)
    const real* xq;    // [K][Nq]   (forcing only)
    const real* yq;
    // FP64 unique-pair schedule: the metric-averaged skew operator entries
    // (Qskew^x, Qskew^y)[j][m] of the pair each lane takes in each step,
    // [K][NSTEP][32][2] (zero where the lane has no pair); stage-independent,
    // formed once on the host
    const real* qxy;
    // FP64 path with the stored inverse (Np <= 16, Nh <= 32): per-element
    // products of the inverse mass with the shared operators, formed once on
    // the host, in the order the lanes read them (zero-padded):
    //   lk [K][(Nh+1)/2][32]  M^-1 Vh^T   (lift + inverse mass), lane = n + 16 hf,
    //                          column l = hf (Nh+1)/2 + t at step t
    //   gk [K][(Nq+1)/2][32]  M^-1 Vq^T   (forcing), the same with columns q
    //   pk [K][Nq][32]        Vh M^-1 Vq^T (projection to the hybrid nodes), lane = l
    // null: the inverse applied to the shared operators' results in turn
    const real* lk;
    const real* gk;
    const real* pk;
    // state
    const double* u_in;  // [3][K][Np]  (projection input)
    double* u;           // [3][K][Np]  RK state (updated in place)
    double* res;         // [3][K][Np]  RK residual
    double* rhs_out;     // [3][K][Np]  RHS mode output
    double* u_out;       // [3][K][Np]  if set: the stage's new state also written here (host-state calls)
    int copy_in;         // projection of u_in: also store u_in into u and zero res
    const real* ut_in;   // [K][Nh][4]  entropy-projected (h, u, v, H) of this stage (the FP32 batched
                         //             kernel k_stage2 stores H - H_0, H_0 the element's H at node 0)
    real* ut_out;        // [K][Nh][4]  ... of the next stage
    double rkA, rkB, dt, t;
    int forcing;
    real mms_amp, mms_bamp, mms_u0, mms_v0;
    int* status;
};

template <typename real>
struct V2;
template <>
struct V2<float> { typedef float2 t; };
template <>
struct V2<double> { typedef double2 t; };

template <typename real>
__device__ __forceinline__ real r_sqrt(real x);
template <>
__device__ __forceinline__ float r_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double r_sqrt<double>(double x) { return sqrt(x); }

template <typename real>
__device__ __forceinline__ void r_sincospi(real x, real* s, real* c);
template <>
__device__ __forceinline__ void r_sincospi<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <>
__device__ __forceinline__ void r_sincospi<double>(double x, double* s, double* c) { sincospi(x, s, c); }

template <typename real>
__device__ __forceinline__ bool r_finite(real x) { return isfinite(x); }

// Row r of a three-field contraction with T terms, for R <= 16 rows: the two
// half-warps take half of the terms each and the sums meet by a shuffle, so
// all 32 lanes work (rows r = lane & 15).  acc(r, t, a0, a1, a2) adds term t.
// Every lane of the warp calls it; it returns true on lanes 0..R-1, which hold
// the sums of row r = lane.
template <int R, int T, typename real, typename Acc>
__device__ __forceinline__ bool split_rows(int lane, Acc acc, real& a0, real& a1, real& a2) {
    static_assert(R <= 16, "two half-warps of rows");
    constexpr int TH = (T + 1) / 2;
    const int r = lane & 15, hf = lane >> 4;
    a0 = a1 = a2 = real(0);
    if (r < R) {
#pragma unroll
        for (int tt = 0; tt < TH; ++tt) {
            const int t = hf * TH + tt;
            if (t < T) acc(r, t, a0, a1, a2);
        }
    }
    a0 += __shfl_down_sync(0xffffffffu, a0, 16);
    a1 += __shfl_down_sync(0xffffffffu, a1, 16);
    a2 += __shfl_down_sync(0xffffffffu, a2, 16);
    return lane < R;
}

// Shared-memory layout of one CTA: reference operators, then one slab per warp.
template <int N, typename real>
struct Smem {
    typedef Dims<N> D;
    static constexpr int REC = 12;  // h hu hv u v H rx sx ry sy 2gh b
    static constexpr int ops_QsT = 0;
    static constexpr int ops_Vq = ops_QsT + D::Nh * D::Nh * 2;
    static constexpr int ops_VqT = ops_Vq + D::Nq * D::Np;
    static constexpr int ops_Vh = ops_VqT + D::Np * D::Nq;
    static constexpr int ops_VhT = ops_Vh + D::Nh * D::Np;
    static constexpr int ops_wf = ops_VhT + D::Np * D::Nh;
    static constexpr int ops_nrs = ops_wf + D::Nfq;
    static constexpr int ops_wq = ops_nrs + 2 * D::Nfq;
    static constexpr int ops_end = ((ops_wq + D::Nq) + 3) & ~3;
    // per-warp slab
    static constexpr int w_rec = 0;                              // [Nh][REC]
    static constexpr int w_rt = w_rec + D::Nh * REC;             // [3][Nh]
    static constexpr int w_a = w_rt + 3 * D::Nh;                 // [3][Nq]
    static constexpr int w_b = w_a + 3 * D::Nq;                  // [3][Np]
    static constexpr int w_c = w_b + 3 * D::Np;                  // [3][Np]
    static constexpr int w_minv = w_c + 3 * D::Np;               // [NpP] (stored inverse only)
    // pair loop of the rules too large for the half-warp split (see k_stage):
    // the NPAIR non-zero pairs, row-major, cut into 32 pieces of PL, each piece
    // touching at most PR rows; partial row sums in w_part [32][PR][4]
    static constexpr bool PIECES = !(D::Nq <= 16 && D::Nh <= 32);
    static constexpr int NPAIR = D::Nq * D::Nh + D::Nfq * D::Nq;
    static constexpr int PL = (NPAIR + 31) / 32;
    static constexpr int PR = (PL + D::Nq - 2) / D::Nq + 1;
    static constexpr int w_part = ((w_minv + (D::wadg ? 0 : D::NpP)) + 3) & ~3;
    static constexpr int w_end = ((w_part + (PIECES ? 32 * PR * 4 : 0)) + 3) & ~3;
    static constexpr size_t bytes(int warps) { return sizeof(real) * (size_t(ops_end) + size_t(warps) * w_end); }
};

template <int N, typename real>
__device__ __forceinline__ void stage_ops_to_smem(const StageParams<real>& p, real* sm) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    for (int i = threadIdx.x; i < D::Nh * D::Nh * 2; i += blockDim.x) sm[S::ops_QsT + i] = p.QsT[i];
    for (int i = threadIdx.x; i < D::Nq * D::Np; i += blockDim.x) {
        sm[S::ops_Vq + i] = p.Vq[i];
        sm[S::ops_VqT + i] = p.VqT[i];
    }
    for (int i = threadIdx.x; i < D::Nh * D::Np; i += blockDim.x) {
        sm[S::ops_Vh + i] = p.Vh[i];
        sm[S::ops_VhT + i] = p.VhT[i];
    }
    for (int i = threadIdx.x; i < D::Nfq; i += blockDim.x) {
        sm[S::ops_wf + i] = p.wf[i];
        sm[S::ops_nrs + 2 * i] = p.nrs[2 * i];
        sm[S::ops_nrs + 2 * i + 1] = p.nrs[2 * i + 1];
    }
    for (int i = threadIdx.x; i < D::Nq; i += blockDim.x) sm[S::ops_wq + i] = p.wq[i];
}

// Weight-adjusted inverse mass (Sec. 2.8's alternative to storing the
// inverses): out = Vq^T diag(w / J) Vq y for the three fields of one element,
// y and out [3][Np] (may alias), t [3][Nq] scratch.
template <int N, typename real>
__device__ __forceinline__ void wadg_apply(const StageParams<real>& p, const real* ops, const real* y, real* t,
                                           real* out, int e, int lane, real sign) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    const real* Vq = ops + S::ops_Vq;
    const real* VqT = ops + S::ops_VqT;
    for (int q = lane; q < D::Nq; q += 32) {
        real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int n = 0; n < D::Np; ++n) {
            const real v = Vq[q * D::Np + n];
            a0 += v * y[n];
            a1 += v * y[D::Np + n];
            a2 += v * y[2 * D::Np + n];
        }
        const real w = ops[S::ops_wq + q];
        const real sc = w * w / p.wJq[(size_t)e * D::Nq + q];
        t[q] = a0 * sc;
        t[D::Nq + q] = a1 * sc;
        t[2 * D::Nq + q] = a2 * sc;
    }
    __syncwarp();
    for (int n = lane; n < D::Np; n += 32) {
        real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
        for (int q = 0; q < D::Nq; ++q) {
            const real v = VqT[n * D::Nq + q];
            a0 += v * t[q];
            a1 += v * t[D::Nq + q];
            a2 += v * t[2 * D::Nq + q];
        }
        out[n] = sign * a0;
        out[D::Np + n] = sign * a1;
        out[2 * D::Np + n] = sign * a2;
    }
}

// Entropy projection of one element's modal state (in w_b, FP `real`) into
// u~ at the hybrid nodes, written to ut_out[e] (Sec. 2.6, J-weighted, Sec. 2.7).
template <int N, typename real>
__device__ __forceinline__ void project_element(const StageParams<real>& p, const real* ops, real* ws, int e,
                                                int lane) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    const real* Vq = ops + S::ops_Vq;
    const real* VqT = ops + S::ops_VqT;
    const real* Vh = ops + S::ops_Vh;
    real* us = ws + S::w_b;     // [3][Np] modal state
    real* ta = ws + S::w_a;     // [3][Nq]
    real* tc = ws + S::w_c;     // [3][Np]
    real* mi = ws + S::w_minv;  // [NpP]
    const real g = p.g;
    int bad = 0;
    // u_q = Vq u_h, v_q = v(u_q), scaled by w_q J_q
    auto vq_term = [&](int q, int n, real& a0, real& a1, real& a2) {
        const real v = Vq[q * D::Np + n];
        a0 += v * us[n];
        a1 += v * us[D::Np + n];
        a2 += v * us[2 * D::Np + n];
    };
    for (int q0 = 0; q0 < D::Nq; q0 += 32) {
        real a0 = 0, a1 = 0, a2 = 0;
        const int q = q0 + lane;
        if constexpr (D::Nq <= 16) {
            if (!split_rows<D::Nq, D::Np>(lane, vq_term, a0, a1, a2)) continue;
        } else {
            if (q >= D::Nq) continue;
#pragma unroll
            for (int n = 0; n < D::Np; ++n) vq_term(q, n, a0, a1, a2);
        }
        real h = a0;
        if (!(h > real(0))) bad |= STATUS_NONPOSITIVE;
        real ih = real(1) / h;
        real uu = a1 * ih, vv = a2 * ih;
        real b = p.bh[(size_t)e * D::Nh + q];
        real w = p.wJq[(size_t)e * D::Nq + q];
        ta[q] = w * (g * (h + b) - real(0.5) * (uu * uu + vv * vv));
        ta[D::Nq + q] = w * uu;
        ta[2 * D::Nq + q] = w * vv;
    }
    __syncwarp();
    // u~ = u(v~) at hybrid node l from v~ = (a0, a1, a2):
    // H = (v1 + (v2^2 + v3^2)/2)/g, h = H - b
    const real ig = real(1) / g;
    auto emit = [&](int l, real a0, real a1, real a2) {
        real H = (a0 + real(0.5) * (a1 * a1 + a2 * a2)) * ig;
        real h = H - p.bh[(size_t)e * D::Nh + l];
        if (!(h > real(0))) bad |= STATUS_NONPOSITIVE;
        if (!r_finite(H) || !r_finite(a1) || !r_finite(a2)) bad |= STATUS_NONFINITE;
        real* o = p.ut_out + ((size_t)e * D::Nh + l) * 4;
        o[0] = h;
        o[1] = a1;
        o[2] = a2;
        o[3] = H;
    };
    if constexpr (!D::wadg && D::Np <= 16 && D::Nh <= 32) {
        if (p.pk != nullptr) {
            // v~ = (Vh M^-1 Vq^T) (W J v_q), the product stored per element; lane = l
            const real* Pk = p.pk + (size_t)e * D::Nq * 32 + lane;
            real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
            for (int q = 0; q < D::Nq; ++q) {
                const real v = Pk[32 * q];
                a0 += v * ta[q];
                a1 += v * ta[D::Nq + q];
                a2 += v * ta[2 * D::Nq + q];
            }
            if (lane < D::Nh) emit(lane, a0, a1, a2);
            if (bad) atomicOr(p.status, bad);
            return;
        }
    }
    // y = Vq^T W J v_q
    auto vqt_term = [&](int n, int q, real& a0, real& a1, real& a2) {
        const real v = VqT[n * D::Nq + q];
        a0 += v * ta[q];
        a1 += v * ta[D::Nq + q];
        a2 += v * ta[2 * D::Nq + q];
    };
    for (int n0 = 0; n0 < D::Np; n0 += 32) {
        real a0 = 0, a1 = 0, a2 = 0;
        const int n = n0 + lane;
        if constexpr (D::Np <= 16) {
            if (!split_rows<D::Np, D::Nq>(lane, vqt_term, a0, a1, a2)) continue;
        } else {
            if (n >= D::Np) continue;
#pragma unroll 5
            for (int q = 0; q < D::Nq; ++q) vqt_term(n, q, a0, a1, a2);
        }
        tc[n] = a0;
        tc[D::Np + n] = a1;
        tc[2 * D::Np + n] = a2;
    }
    __syncwarp();
    if constexpr (D::wadg) {
        // v_h = Vq^T diag(w / J) Vq y  (weight-adjusted inverse; ta is free again)
        wadg_apply<N, real>(p, ops, tc, ta, us, e, lane, real(1));
    } else {
        // v_h = (M_h^k)^{-1} y   (packed symmetric)
        auto mi_term = [&](int n, int j, real& a0, real& a1, real& a2) {
            const int ij = n >= j ? n * (n + 1) / 2 + j : j * (j + 1) / 2 + n;
            const real m = mi[ij];
            a0 += m * tc[j];
            a1 += m * tc[D::Np + j];
            a2 += m * tc[2 * D::Np + j];
        };
        for (int n0 = 0; n0 < D::Np; n0 += 32) {
            real a0 = 0, a1 = 0, a2 = 0;
            const int n = n0 + lane;
            if constexpr (D::Np <= 16) {
                if (!split_rows<D::Np, D::Np>(lane, mi_term, a0, a1, a2)) continue;
            } else {
                if (n >= D::Np) continue;
#pragma unroll
                for (int j = 0; j < D::Np; ++j) mi_term(n, j, a0, a1, a2);
            }
            us[n] = a0;   // us is free again: reuse for v_h
            us[D::Np + n] = a1;
            us[2 * D::Np + n] = a2;
        }
    }
    __syncwarp();
    // v~ = Vh v_h, then u~ = u(v~)
    for (int l = lane; l < D::Nh; l += 32) {
        real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
        for (int n = 0; n < D::Np; ++n) {
            real v = Vh[l * D::Np + n];
            a0 += v * us[n];
            a1 += v * us[D::Np + n];
            a2 += v * us[2 * D::Np + n];
        }
        emit(l, a0, a1, a2);
    }
    if (bad) atomicOr(p.status, bad);
}

template <int N, typename real>
__device__ __forceinline__ void load_minv(const StageParams<real>& p, real* ws, int e, int lane) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    // (not read where the products with the inverse are stored)
    if constexpr (!D::wadg)
        if (p.pk == nullptr)
            for (int i = lane; i < D::NpP; i += 32) ws[S::w_minv + i] = p.minv[(size_t)e * p.mstride + i];
}

// Standalone projection: u_in (FP64 modal) -> ut_out.
template <int N, typename real>
__global__ void __launch_bounds__(256) k_project(StageParams<real> p) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* ops = reinterpret_cast<real*>(smem_raw);
    stage_ops_to_smem<N, real>(p, ops);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    real* ws = ops + S::ops_end + warp * S::w_end;
    for (int e = blockIdx.x * wpb + warp; e < p.K; e += gridDim.x * wpb) {
        load_minv<N, real>(p, ws, e, lane);
        for (int i = lane; i < 3 * D::Np; i += 32) {
            int c = i / D::Np, n = i - c * D::Np;
            const size_t gi = ((size_t)c * p.K + e) * D::Np + n;
            const double un = p.u_in[gi];
            ws[S::w_b + i] = (real)un;
            if (p.copy_in) {
                p.u[gi] = un;
                p.res[gi] = 0.0;
            }
        }
        __syncwarp();
        project_element<N, real>(p, ops, ws, e, lane);
        __syncwarp();
    }
}

// MODE 0: write du/dt to rhs_out.  MODE 1: LSRK45 stage update of (u, res)
// followed by the entropy projection of the new state into ut_out.
template <int N, typename real, int MODE>
__device__ __forceinline__ void k_stage_body(const StageParams<real>& p) {
    typedef Dims<N> D;
    typedef Smem<N, real> S;
    typedef typename V2<real>::t real2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* ops = reinterpret_cast<real*>(smem_raw);
    stage_ops_to_smem<N, real>(p, ops);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    real* ws = ops + S::ops_end + warp * S::w_end;
    real* rec = ws + S::w_rec;
    real* rt = ws + S::w_rt;
    const real2* QsT = reinterpret_cast<const real2*>(ops + S::ops_QsT);
    const real g = p.g;
    const real eighth = real(0.125);

    for (int e = blockIdx.x * wpb + warp; e < p.K; e += gridDim.x * wpb) {
        // ---- load u~ and geometry of the element -------------------------------
        for (int l = lane; l < D::Nh; l += 32) {
            const real* ut = p.ut_in + ((size_t)e * D::Nh + l) * 4;
            const real* gg = p.geo + ((size_t)e * D::Nh + l) * 4;
            real h = ut[0], uu = ut[1], vv = ut[2], H = ut[3];
            real* r = rec + l * S::REC;
            r[0] = h;
            r[1] = h * uu;
            r[2] = h * vv;
            r[3] = uu;
            r[4] = vv;
            r[5] = H;
            r[6] = gg[0] * eighth;
            r[7] = gg[1] * eighth;
            r[8] = gg[2] * eighth;
            r[9] = gg[3] * eighth;
            r[10] = real(2) * g * h;
            r[11] = H - h;
        }
        load_minv<N, real>(p, ws, e, lane);
        __syncwarp();
        // ---- volume flux differencing + interface flux, row l = lane ----------
        // (u_l + u_m) T summed over m is u_l (sum of T) + sum of u_m T: the row
        // part is added once after the pair loop.
        //
        // With Nq <= 16 and Nh <= 32 every non-zero pair (l, m) of Q_skew is
        // evaluated once (the face-face block is zero): the flux terms are
        // antisymmetric in (l, m) (T_ml = -T_lm) and the pressure terms swap
        // h and H, so one evaluation gives row l its contribution and row m
        // -(u_l T + Qx g h_m H_l), ... (with the stored metric-averaged entries,
        // 17 FP64 instructions for both rows, the receiver's three subtractions
        // included: this kernel is bound by the FP64 pipe).  Lanes
        // j = lane & 15 of half-warp hf stand for volume row j.  Volume-volume
        // pairs run along the diagonals (j, j + d mod Nq), volume-face pairs
        // along (j, Nq + (j + t) mod L), L = max(Nq, Nfq), the two half-warps
        // splitting the diagonals; in every step each row receives exactly one
        // transposed contribution, from the lane d (or t) places before it,
        // by a shuffle.  The half-warps' partial sums meet at the end.
        constexpr bool SPLIT = D::Nq <= 16 && D::Nh <= 32;
        real tl0 = 0, tl1 = 0, tl2 = 0;  // the lane's own row sums after the pair loop
        if constexpr (SPLIT) {
            typedef PairSched<N> PS;
            constexpr int V = PS::V, F = PS::F, L = PS::L;
            static_assert(L <= 16, "one half-warp per diagonal");
            constexpr int SVV = PS::SVV;          // volume-volume diagonals d = 1..SVV
            constexpr int SVV0 = PS::SVV0;        // half 0: d = 1..SVV0, half 1: d = SVV0+1..SVV
            constexpr int SVF0 = PS::SVF0;        // volume-face: half 0: t < SVF0, half 1: the rest
            // this lane's stored operator entries, one (Qx, Qy) per step
            const real* qe = p.qxy + ((size_t)e * PS::NSTEP * 32 + lane) * 2;
            const int j = lane & 15, hf = lane >> 4;
            const bool vrow = j < V;
            const real* rl = rec + (vrow ? j : 0) * S::REC;
            const real h_l = rl[0], hu_l = rl[1], hv_l = rl[2], u_l = rl[3], v_l = rl[4], H_l = rl[5];
            const real gh2_l = rl[10];
            real A0 = 0, A1 = 0, A2 = 0;  // volume row j: own side + transposed volume-volume terms
            real A1p = 0, A2p = 0;        // volume row j: sum of (Qx, Qy) H_m, times 2 g h_j after the loop
            real B0 = 0, B1 = 0, B2 = 0;  // face row Nq + j: transposed volume-face terms
            // pair (j, m): own-row terms into (A0, A1, A2, A1p, A2p), the row-m
            // terms, to be subtracted by their receiver, into (t0, t1, t2)
            auto pair = [&](int m, real Qx, real Qy, real& t0, real& t1, real& t2) {
                const real* rm = rec + m * S::REC;
                const real HU = hu_l + rm[1], HV = hv_l + rm[2];
                const real T = Qx * HU + Qy * HV;
                const real Pml = rm[10] * H_l;      // 2 g h_m H_l
                A0 += T;
                A1 = fma(rm[3], T, A1);
                A2 = fma(rm[4], T, A2);
                A1p = fma(Qx, rm[5], A1p);
                A2p = fma(Qy, rm[5], A2p);
                t0 = T;
                t1 = fma(u_l, T, Qx * Pml);
                t2 = fma(v_l, T, Qy * Pml);
            };
#pragma unroll
            for (int k = 0; k < SVV0; ++k) {
                const int d = hf == 0 ? 1 + k : SVV0 + 1 + k;
                const bool step = d <= SVV;
                // for d = V / 2 both ends of a pair are d apart: the lower half of the rows takes it
                const bool act = vrow && step && !(2 * d == V && j >= V / 2);
                int m = j + d;
                m -= m >= V ? V : 0;
                const real2 q = *reinterpret_cast<const real2*>(qe + 64 * k);
                real t0 = 0, t1 = 0, t2 = 0;
                if (act) pair(m, q.x, q.y, t0, t1, t2);
                int src = j - d;
                src += src < 0 ? V : 0;
                const real r0 = __shfl_sync(0xffffffffu, t0, 16 * hf + (src & 15));
                const real r1 = __shfl_sync(0xffffffffu, t1, 16 * hf + (src & 15));
                const real r2 = __shfl_sync(0xffffffffu, t2, 16 * hf + (src & 15));
                if (vrow && step) {
                    A0 -= r0;
                    A1 -= r1;
                    A2 -= r2;
                }
            }
#pragma unroll
            for (int k = 0; k < SVF0; ++k) {
                const int t = hf == 0 ? k : SVF0 + k;
                const bool step = t < L;
                int f = j + t;
                f -= f >= L ? L : 0;
                const bool act = vrow && step && f < F;
                const real2 q = *reinterpret_cast<const real2*>(qe + 64 * (SVV0 + k));
                real t0 = 0, t1 = 0, t2 = 0;
                if (act) pair(V + f, q.x, q.y, t0, t1, t2);
                int src = j - t;
                src += src < 0 ? L : 0;
                const real r0 = __shfl_sync(0xffffffffu, t0, 16 * hf + (src & 15));
                const real r1 = __shfl_sync(0xffffffffu, t1, 16 * hf + (src & 15));
                const real r2 = __shfl_sync(0xffffffffu, t2, 16 * hf + (src & 15));
                if (step && j < F) {
                    B0 -= r0;
                    B1 -= r1;
                    B2 -= r2;
                }
            }
            A1 = fma(gh2_l, A1p, A1);  // the pressure terms g h_j H_m of row j's own pairs
            A2 = fma(gh2_l, A2p, A2);
            A0 += __shfl_xor_sync(0xffffffffu, A0, 16);
            A1 += __shfl_xor_sync(0xffffffffu, A1, 16);
            A2 += __shfl_xor_sync(0xffffffffu, A2, 16);
            B0 += __shfl_xor_sync(0xffffffffu, B0, 16);
            B1 += __shfl_xor_sync(0xffffffffu, B1, 16);
            B2 += __shfl_xor_sync(0xffffffffu, B2, 16);
            // face row Nq + i lives on lane Nq + i: fetch B of lane i
            const int fsrc = (lane - V) & 31;
            const real b0 = __shfl_sync(0xffffffffu, B0, fsrc);
            const real b1 = __shfl_sync(0xffffffffu, B1, fsrc);
            const real b2 = __shfl_sync(0xffffffffu, B2, fsrc);
            if (lane < V) {
                tl0 = A0; tl1 = A1; tl2 = A2;
            } else if (lane < D::Nh) {
                tl0 = b0; tl1 = b1; tl2 = b2;
            }
            (void)h_l;
        }
        // Larger rules: the non-zero pairs (volume rows x Nh columns, then face
        // rows x Nq columns), row-major, in 32 equal pieces, one per lane; a
        // piece files its partial row sums when a row ends, and each row's
        // owner adds up the pieces of its row below.
        real* part = ws + S::w_part;
        if constexpr (S::PIECES) {
            const int p0 = lane * S::PL;
            const int p1 = p0 + S::PL < S::NPAIR ? p0 + S::PL : S::NPAIR;
            const int pp = p0 < p1 ? p0 : 0;
            int r, m, len, slot = 0;
            if (pp < D::Nq * D::Nh) {
                r = pp / D::Nh;
                m = pp - r * D::Nh;
                len = D::Nh;
            } else {
                const int q = pp - D::Nq * D::Nh;
                r = D::Nq + q / D::Nq;
                m = q - (r - D::Nq) * D::Nq;
                len = D::Nq;
            }
            const real* rl = rec + r * S::REC;
            real hu_l = rl[1], hv_l = rl[2], rx_l = rl[6], sx_l = rl[7], ry_l = rl[8], sy_l = rl[9], gh2_l = rl[10];
            real c0 = 0, c1 = 0, c2 = 0;
            for (int k = 0; k < S::PR * 4; ++k) part[lane * S::PR * 4 + k] = real(-1);
#pragma unroll 1
            for (int it = 0; it < S::PL; ++it) {
                if (p0 + it < p1) {
                    const real2 q = QsT[m * D::Nh + r];
                    const real* rm = rec + m * S::REC;
                    const real Qx = q.x * (rx_l + rm[6]) + q.y * (sx_l + rm[7]);
                    const real Qy = q.x * (ry_l + rm[8]) + q.y * (sy_l + rm[9]);
                    const real HU = hu_l + rm[1], HV = hv_l + rm[2];
                    const real T = Qx * HU + Qy * HV;
                    const real P = gh2_l * rm[5];
                    c0 += T;
                    c1 = fma(rm[3], T, fma(Qx, P, c1));
                    c2 = fma(rm[4], T, fma(Qy, P, c2));
                    if (++m == len || p0 + it + 1 == p1) {
                        real* o = part + (lane * S::PR + slot) * 4;
                        o[0] = c0;
                        o[1] = c1;
                        o[2] = c2;
                        o[3] = real(r);
                        ++slot;
                        c0 = c1 = c2 = 0;
                        if (m == len && r + 1 < D::Nh) {
                            ++r;
                            m = 0;
                            len = r < D::Nq ? D::Nh : D::Nq;
                            rl = rec + r * S::REC;
                            hu_l = rl[1]; hv_l = rl[2]; rx_l = rl[6]; sx_l = rl[7]; ry_l = rl[8]; sy_l = rl[9];
                            gh2_l = rl[10];
                        }
                    }
                }
            }
            __syncwarp();
        }
        // Lax-Friedrichs wave speeds |u.nJ| + sqrt(sJ^2 g h) (the unit normal
        // n = nJ / sJ folded in) of both sides of every face node in one pass
        // over the warp, where the face rows sit on lanes Nq.. = 16..: lane
        // 16 + f takes face node f's own trace, lane f the neighbour's (a wall
        // mirrors the normal velocity and keeps h, so its speed is the own one);
        // face row Nq + f then reads the neighbour's speed from lane f.
        constexpr bool LF_PAIRED = SPLIT && D::Nq == 16 && D::Nfq <= 16;
        real lam_pass = 0;
        if constexpr (LF_PAIRED) {
            __syncwarp();
            const int f = lane & 15;
            if (p.lf && f < D::Nfq) {
                const real* rf = rec + (D::Nq + f) * S::REC;
                const real nr = ops[S::ops_nrs + 2 * f], ns = ops[S::ops_nrs + 2 * f + 1];
                const real fx = real(8) * (rf[6] * nr + rf[7] * ns);
                const real fy = real(8) * (rf[8] * nr + rf[9] * ns);
                real hh = rf[0], uu = rf[3], vv = rf[4];
                if (lane < 16) {
                    const int face = f / D::Nfp, i = f - face * D::Nfp;
                    const int nb = p.nbr[(size_t)e * 3 + face];
                    if ((nb & 3) != 3) {
                        const real* up =
                            p.ut_in + ((size_t)(nb >> 2) * D::Nh + D::Nq + (nb & 3) * D::Nfp + (D::Nfp - 1 - i)) * 4;
                        hh = up[0];
                        uu = up[1];
                        vv = up[2];
                    }
                }
                lam_pass = fabs(uu * fx + vv * fy) + r_sqrt((fx * fx + fy * fy) * g * hh);
            }
        }
        const real lam_nbr = LF_PAIRED ? __shfl_sync(0xffffffffu, lam_pass, lane & 15) : real(0);
        for (int l = lane; l < D::Nh; l += 32) {
            const real* rl = rec + l * S::REC;
            const real h_l = rl[0], hu_l = rl[1], hv_l = rl[2], u_l = rl[3], v_l = rl[4];
            const real rx_l = rl[6], sx_l = rl[7], ry_l = rl[8], sy_l = rl[9];
            real a0 = 0, a1 = 0, a2 = 0;
            if constexpr (SPLIT) {
                a0 = tl0;
                a1 = tl1;
                a2 = tl2;
            } else {
                // the pieces of row l, in lane order
                const int start = l < D::Nq ? l * D::Nh : D::Nq * D::Nh + (l - D::Nq) * D::Nq;
                const int len = l < D::Nq ? D::Nh : D::Nq;
                const int k0 = start / S::PL, k1 = (start + len - 1) / S::PL;
                for (int k = k0; k <= k1; ++k)
#pragma unroll
                    for (int sl = 0; sl < S::PR; ++sl) {
                        const real* o = part + (k * S::PR + sl) * 4;
                        if (o[3] == real(l)) {
                            a0 += o[0];
                            a1 += o[1];
                            a2 += o[2];
                        }
                    }
            }
            a1 += u_l * a0;
            a2 += v_l * a0;
            real r0 = real(2) * a0, r1 = a1, r2 = a2;
            if (l >= D::Nq) {
                // interface: f_S(u~+, u~) with the well-balanced pressure
                // g/2 h (h+ + b), and Lax-Friedrichs on the jump of u~
                const int f = l - D::Nq;
                const int face = f / D::Nfp, i = f - face * D::Nfp;
                const int nb = p.nbr[(size_t)e * 3 + face];
                const int en = nb >> 2, fn = nb & 3;
                const real nr = ops[S::ops_nrs + 2 * f], ns = ops[S::ops_nrs + 2 * f + 1];
                const real nxJ = real(8) * (rx_l * nr + sx_l * ns);
                const real nyJ = real(8) * (ry_l * nr + sy_l * ns);
                real hP, uP, vP;
                if (fn == 3) {
                    // reflective wall (Sec. 2.9): h+ = h, u_n+ = -u_n, tangential kept
                    const real sJw = r_sqrt(nxJ * nxJ + nyJ * nyJ);
                    const real wnx = nxJ / sJw, wny = nyJ / sJw;
                    const real un = u_l * wnx + v_l * wny;
                    hP = h_l;
                    uP = u_l - real(2) * un * wnx;
                    vP = v_l - real(2) * un * wny;
                } else {
                    const real* up = p.ut_in + ((size_t)en * D::Nh + D::Nq + fn * D::Nfp + (D::Nfp - 1 - i)) * 4;
                    hP = up[0];
                    uP = up[1];
                    vP = up[2];
                }
                const real huP = hP * uP, hvP = hP * vP;
                const real w = ops[S::ops_wf + f];
                const real b_l = rl[11];
                const real huA = real(0.5) * (hu_l + huP), hvA = real(0.5) * (hv_l + hvP);
                const real uA = real(0.5) * (u_l + uP), vA = real(0.5) * (v_l + vP);
                const real pw = real(0.5) * g * h_l * (hP + b_l);
                const real Fn0 = nxJ * huA + nyJ * hvA;
                const real Fn1 = uA * Fn0 + nxJ * pw;
                const real Fn2 = vA * Fn0 + nyJ * pw;
                r0 += w * Fn0;
                r1 += w * Fn1;
                r2 += w * Fn2;
                if (p.lf) {
                    // sJ max(|u.n| + sqrt(g h)) over both sides with the unit
                    // normal n = nJ / sJ folded in: |u.nJ| + sqrt(sJ^2 g h)
                    real lm, lp;
                    if constexpr (LF_PAIRED) {
                        lm = lam_pass;  // this lane is 16 + f: its own side, computed above
                        lp = lam_nbr;
                    } else {
                        const real sJ2 = nxJ * nxJ + nyJ * nyJ;
                        lm = fabs(u_l * nxJ + v_l * nyJ) + r_sqrt(sJ2 * g * h_l);
                        lp = fabs(uP * nxJ + vP * nyJ) + r_sqrt(sJ2 * g * hP);
                    }
                    const real c = real(0.5) * w * (lm > lp ? lm : lp);
                    r0 -= c * (hP - h_l);
                    r1 -= c * (huP - hu_l);
                    r2 -= c * (hvP - hv_l);
                }
            }
            rt[l] = r0;
            rt[D::Nh + l] = r1;
            rt[2 * D::Nh + l] = r2;
        }
        // forcing at the volume nodes, J-weighted: added as + Vq^T W J f
        real* fa = ws + S::w_a;
        if (p.forcing) {
            for (int q = lane; q < D::Nq; q += 32) {
                const real x = p.xq[(size_t)e * D::Nq + q], y = p.yq[(size_t)e * D::Nq + q];
                const real w = p.wJq[(size_t)e * D::Nq + q];
                real sth, cth, sx, cx, sy, cy;
                r_sincospi<real>(x + y - real(p.t), &sth, &cth);
                r_sincospi<real>(x, &sx, &cx);
                r_sincospi<real>(y, &sy, &cy);
                const real pi = real(3.14159265358979323846);
                const real h = real(2) + p.mms_amp * sth;
                const real c = p.mms_amp * pi * cth;
                const real ht = -c, hx = c, hy = c;
                const real bx = -p.mms_bamp * pi * sx * cy, by = -p.mms_bamp * pi * cx * sy;
                const real u0 = p.mms_u0, v0 = p.mms_v0;
                fa[q] = w * (ht + u0 * hx + v0 * hy);
                fa[D::Nq + q] = w * (u0 * ht + (u0 * u0 + g * h) * hx + u0 * v0 * hy + g * h * bx);
                fa[2 * D::Nq + q] = w * (v0 * ht + u0 * v0 * hx + (v0 * v0 + g * h) * hy + g * h * by);
            }
        }
        __syncwarp();
        real* sc = ws + S::w_c;
        bool composed = false;
        if constexpr (!D::wadg && D::Np <= 16 && D::Nh <= 32) composed = p.lk != nullptr;
        if (composed) {
            // ---- M^-1 s = (M^-1 Vh^T) r - (M^-1 Vq^T) (W J f), the products stored
            // per element: rows n = lane & 15 over the columns of half-warp hf
            constexpr int LT = (D::Nh + 1) / 2, GT = (D::Nq + 1) / 2;
            const int hf = lane >> 4;
            const real* Lk = p.lk + (size_t)e * LT * 32 + lane;
            real a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
            for (int t = 0; t < LT; ++t) {
                const int l = hf * LT + t;
                if (l < D::Nh) {
                    const real v = Lk[32 * t];
                    a0 += v * rt[l];
                    a1 += v * rt[D::Nh + l];
                    a2 += v * rt[2 * D::Nh + l];
                }
            }
            if (p.forcing) {
                const real* Gk = p.gk + (size_t)e * GT * 32 + lane;
#pragma unroll
                for (int t = 0; t < GT; ++t) {
                    const int q = hf * GT + t;
                    if (q < D::Nq) {
                        const real v = Gk[32 * t];
                        a0 -= v * fa[q];
                        a1 -= v * fa[D::Nq + q];
                        a2 -= v * fa[2 * D::Nq + q];
                    }
                }
            }
            a0 += __shfl_down_sync(0xffffffffu, a0, 16);
            a1 += __shfl_down_sync(0xffffffffu, a1, 16);
            a2 += __shfl_down_sync(0xffffffffu, a2, 16);
            if (lane < D::Np) {
                sc[lane] = a0;
                sc[D::Np + lane] = a1;
                sc[2 * D::Np + lane] = a2;
            }
        } else {
        // ---- lift: s = Vh^T r - Vq^T W J f --------------------------------------
        const real* VhT = ops + S::ops_VhT;
        const real* VqT = ops + S::ops_VqT;
        real* sb = ws + S::w_b;
        auto vht_term = [&](int n, int l, real& a0, real& a1, real& a2) {
            const real v = VhT[n * D::Nh + l];
            a0 += v * rt[l];
            a1 += v * rt[D::Nh + l];
            a2 += v * rt[2 * D::Nh + l];
        };
        auto frc_term = [&](int n, int q, real& a0, real& a1, real& a2) {
            const real v = VqT[n * D::Nq + q];
            a0 -= v * fa[q];
            a1 -= v * fa[D::Nq + q];
            a2 -= v * fa[2 * D::Nq + q];
        };
        for (int n0 = 0; n0 < D::Np; n0 += 32) {
            real a0 = 0, a1 = 0, a2 = 0;
            const int n = n0 + lane;
            if constexpr (D::Np <= 16) {
                const bool own = split_rows<D::Np, D::Nh>(lane, vht_term, a0, a1, a2);
                if (p.forcing) {
                    real f0, f1, f2;
                    split_rows<D::Np, D::Nq>(lane, frc_term, f0, f1, f2);
                    a0 += f0;
                    a1 += f1;
                    a2 += f2;
                }
                if (!own) continue;
            } else {
                if (n >= D::Np) continue;
#pragma unroll 8
                for (int l = 0; l < D::Nh; ++l) vht_term(n, l, a0, a1, a2);
                if (p.forcing)
                    for (int q = 0; q < D::Nq; ++q) frc_term(n, q, a0, a1, a2);
            }
            sb[n] = a0;
            sb[D::Np + n] = a1;
            sb[2 * D::Np + n] = a2;
        }
        __syncwarp();
        // ---- du/dt = -(M_h^k)^{-1} s; then output or RK update --------------------
        if constexpr (D::wadg) {
            wadg_apply<N, real>(p, ops, sb, fa, sc, e, lane, real(1));  // fa (forcing) is consumed
        } else {
            const real* mi = ws + S::w_minv;
            auto mi_term = [&](int n, int j, real& a0, real& a1, real& a2) {
                const int ij = n >= j ? n * (n + 1) / 2 + j : j * (j + 1) / 2 + n;
                const real m = mi[ij];
                a0 += m * sb[j];
                a1 += m * sb[D::Np + j];
                a2 += m * sb[2 * D::Np + j];
            };
            for (int n0 = 0; n0 < D::Np; n0 += 32) {
                real a0 = 0, a1 = 0, a2 = 0;
                const int n = n0 + lane;
                if constexpr (D::Np <= 16) {
                    if (!split_rows<D::Np, D::Np>(lane, mi_term, a0, a1, a2)) continue;
                } else {
                    if (n >= D::Np) continue;
#pragma unroll
                    for (int j = 0; j < D::Np; ++j) mi_term(n, j, a0, a1, a2);
                }
                sc[n] = a0;
                sc[D::Np + n] = a1;
                sc[2 * D::Np + n] = a2;
            }
        }
        }
        __syncwarp();
        for (int i = lane; i < 3 * D::Np; i += 32) {
            const int c = i / D::Np, n = i - c * D::Np;
            const size_t gi = ((size_t)c * p.K + e) * D::Np + n;
            const double r = (double)sc[i];  // du/dt = -r
            if (MODE == 0) {
                p.rhs_out[gi] = -r;
            } else {
                const double rs = p.rkA * p.res[gi] - p.dt * r;
                p.res[gi] = rs;
                const double un = p.u[gi] + p.rkB * rs;
                p.u[gi] = un;
                if (p.u_out) p.u_out[gi] = un;
                ws[S::w_b + i] = (real)un;  // the projection's input
            }
        }
        __syncwarp();
        if (MODE == 1) {
            project_element<N, real>(p, ops, ws, e, lane);
            __syncwarp();
        }
    }
}

template <int N, typename real, int MODE>
__global__ void __launch_bounds__(256) k_stage(StageParams<real> p) {
    k_stage_body<N, real, MODE>(p);
}

// The same kernel with a floor of MINB blocks of 8 warps per SM for the
// register allocator: the RK stage of N = 4 with the 16-point rule and the
// stored inverse compiles to 127 registers and 2 blocks under the plain bound,
// to 80 and 3 blocks with MINB = 3 (3.34 against 3.41 ms per stage at
// K = 131072); elsewhere the plain bound's allocation is kept (an explicit
// floor makes the allocator fill up to it, and a cap at 80 spills).
template <int N, typename real, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) k_stage(StageParams<real> p) {
    k_stage_body<N, real, MODE>(p);
}

template <int N, int MODE>
constexpr bool k_stage_three_blocks() {
    return MODE == 1 && Dims<N>::Nq == 16 && Dims<N>::Nh == 31 && !Dims<N>::wadg;
}

// FP64 diagnostics: per-CTA partial sums of (entropy, mass, entropy rate).
template <int N>
__global__ void __launch_bounds__(256) k_entropy(int K, double g, const double* __restrict__ u,
                                                 const double* __restrict__ rhs, const double* __restrict__ Vq,
                                                 const double* __restrict__ wJq, const double* __restrict__ bq,
                                                 double* __restrict__ partial) {
    typedef Dims<N> D;
    double s_ent = 0, s_mass = 0, s_rate = 0;
    const size_t total = (size_t)K * D::Nq;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx / D::Nq), q = (int)(idx - (size_t)e * D::Nq);
        double a[3] = {0, 0, 0}, d[3] = {0, 0, 0};
        for (int n = 0; n < D::Np; ++n) {
            const double v = Vq[q * D::Np + n];
            for (int c = 0; c < 3; ++c) {
                a[c] += v * u[((size_t)c * K + e) * D::Np + n];
                if (rhs) d[c] += v * rhs[((size_t)c * K + e) * D::Np + n];
            }
        }
        const double w = wJq[idx], b = bq[idx];
        const double h = a[0], uu = a[1] / h, vv = a[2] / h;
        s_ent += w * (0.5 * (a[1] * uu + a[2] * vv) + 0.5 * g * h * h + g * h * b);
        s_mass += w * h;
        if (rhs) s_rate += w * ((g * (h + b) - 0.5 * (uu * uu + vv * vv)) * d[0] + uu * d[1] + vv * d[2]);
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

// Sum the per-CTA partials in a fixed order (deterministic).
__global__ void k_entropy_finalize(int nparts, const double* __restrict__ partial, double* __restrict__ out);

}  // namespace esdg
