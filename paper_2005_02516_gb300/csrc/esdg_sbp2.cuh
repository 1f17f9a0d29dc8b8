// Batched FP32 DG-SBP stage kernel for sm_103a (right-hand side in FP32, RK
// state in FP64): the operator of k_sbp (esdg_sbp.cuh, Sec. 3) mapped like
// k_stage2 (esdg_stage2.cuh):
//
//  * a warp processes EPW = 4 elements, LPE = 8 lanes per element; lane (e, b)
//    owns the nodes l = b + LPE*i, i < RPL, with their record and three
//    accumulators in registers, so each column m (a node record and the
//    lane's operator entries, float4 reads) feeds RPL rows.  The skew SBP
//    operator is dense (face nodes are volume nodes), so every row takes all
//    Nq columns.
//  * the batch's nodal records (h, u, v, H) and metrics arrive in shared
//    memory by bulk copies (cp.async.bulk) on a per-warp mbarrier with a
//    bounded wait; neighbour values are gathered with plain loads meanwhile.
//  * each lane finishes its own rows: interface flux with Lax-Friedrichs at
//    face nodes, du/dt = -r / (w J) (+ forcing), the LSRK45 stage in FP64 and
//    the next stage's record, without a shared-memory round trip.
#pragma once

#include "esdg_sbp.cuh"
#include "esdg_stage2.cuh"

namespace esdg {

template <int N>
struct S2 {
    typedef SbpDims<N> D;
    static constexpr int LPE = 8;
    static constexpr int EPW = 32 / LPE;
    static constexpr int RPL = (D::Nq + LPE - 1) / LPE;
    // operator entries per (column, lane slot): a multiple of 4 with an odd
    // quotient, so the 8 lanes' float4 reads of one column hit distinct 4-bank groups
    static constexpr int OPB = ((2 * RPL + 3) / 4) % 2 == 1 ? (2 * RPL + 3) / 4 * 4 : (2 * RPL + 3) / 4 * 4 + 4;
    // element slot of the record / metric staging (floats): not 0 or 16 mod 32
    static constexpr int UTS = ((D::Nq * 4 + 4) % 32 == 0 || (D::Nq * 4 + 4) % 32 == 16) ? D::Nq * 4 + 8 : D::Nq * 4 + 4;
    static constexpr int o_Qs = 0;                              // [Nq][LPE][OPB] (Qskew^r, Qskew^s) / 8
    static constexpr int o_wf = o_Qs + D::Nq * LPE * OPB;       // [Nfq]
    static constexpr int o_nrs = o_wf + D::Nfq;                 // [Nfq][2]
    static constexpr int o_fmap = o_nrs + 2 * D::Nfq;           // [Nfq] int: volume node of face node
    static constexpr int o_frow = o_fmap + D::Nfq;              // [Nq]  int: face node of volume node, or -1
    static constexpr int o_end = (o_frow + D::Nq + 3) & ~3;
    static constexpr int w_ut = 0;                              // [EPW][UTS] h u v H
    static constexpr int w_geo = w_ut + EPW * UTS;              // [EPW][UTS] rxJ sxJ ryJ syJ
    static constexpr int w_tr = w_geo + EPW * UTS;              // [EPW][Nfq][4] neighbour values
    static constexpr int w_end = (w_tr + EPW * D::Nfq * 4 + 3) & ~3;
    static constexpr int TRL = (EPW * D::Nfq + 31) / 32;
    static constexpr int SMEM_MAX = 232448;
    static constexpr int WARPS_FIT = (SMEM_MAX - 4 * o_end) / (4 * w_end + 8);
    // at most 24 warps (80 registers a thread) up to 22 nodes (N <= 4), 20 (96
    // registers) above, where 80 registers spill: 24 warps ran 6-11% faster
    // than 16 at 128 registers
    static constexpr int WARPS_CAP = D::Nq <= 22 ? 24 : 20;
    static constexpr int WARPS = WARPS_FIT < WARPS_CAP ? WARPS_FIT : WARPS_CAP;
    static constexpr size_t bytes() { return sizeof(float) * (size_t(o_end) + size_t(WARPS) * w_end) + 8 * WARPS; }
    static constexpr int TX_BYTES = EPW * 2 * D::Nq * 16;
};

template <int N, int MODE>
__device__ __forceinline__ bool sbp2_batch(const StageParams<float>& p, const float* __restrict__ ops, float* ws,
                                           uint64_t* bar, uint32_t& parity, int e0, int lane) {
    typedef SbpDims<N> D;
    typedef S2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const float g = p.g;
    const int K = p.K;
    const int ge = e0 + e;
    const bool valid = ge < K;
    const int* fmap = reinterpret_cast<const int*>(ops + C::o_fmap);
    const int* frow = reinterpret_cast<const int*>(ops + C::o_frow);
    // ---- records and metrics of the batch: bulk copies, one per element and array
    if (lane == 0) mbar_arrive_expect_tx(bar, C::TX_BYTES);
    __syncwarp();
    if (lane < 2 * EPW) {
        const int which = lane / EPW, ee = lane - which * EPW;
        if (which == 0)
            tma_bulk_g2s(ws + C::w_ut + ee * C::UTS, p.ut_in + (size_t)(e0 + ee) * D::Nq * 4, D::Nq * 16, bar);
        else
            tma_bulk_g2s(ws + C::w_geo + ee * C::UTS, p.geo + (size_t)(e0 + ee) * D::Nq * 4, D::Nq * 16, bar);
    }
    // neighbour values at the batch's face nodes (a gather, while the copies fly)
#pragma unroll
    for (int t = 0; t < C::TRL; ++t) {
        const int k = lane + 32 * t;
        if (k < EPW * D::Nfq) {
            const int ee = k / D::Nfq, f = k - ee * D::Nfq;
            const int face = f / D::Nfp, i = f - face * D::Nfp;
            const int nb = __ldg(p.nbr + (size_t)(e0 + ee) * 3 + face);
            const int en = nb >> 2, fn = nb & 3;
            const float4 v = __ldg(reinterpret_cast<const float4*>(
                p.ut_in + ((size_t)en * D::Nq + fmap[fn * D::Nfp + (D::Nfp - 1 - i)]) * 4));
            *reinterpret_cast<float4*>(ws + C::w_tr + k * 4) = v;
        }
    }
    // own operands of the later phases, loaded before the wait (the FP64 RK
    // operands only while they fit the register budget of 24 warps: up to 2
    // rows a lane; loaded late, N = 3, 4 run 24 warps at 78 registers, 3-4%
    // faster than 20 warps with early loads)
    constexpr bool EARLY = RPL <= 2;
    float wj[RPL], bl[RPL];
    double uo[RPL][3], ro[RPL][3];
    auto load_rk = [&](int i) {
        const int l = b + LPE * i;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            uo[i][c] = 0.0;
            ro[i][c] = 0.0;
            if (MODE == 1 && valid && l < D::Nq) {
                const size_t gi = ((size_t)c * K + ge) * D::Nq + l;
                uo[i][c] = p.u[gi];
                if (p.rkA != 0.0) ro[i][c] = p.res[gi];  // the first LSRK45 stage (A = 0) does not read it
            }
        }
    };
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int l = b + LPE * i;
        const bool ok = valid && l < D::Nq;
        wj[i] = ok ? __ldg(p.wJq + (size_t)ge * D::Nq + l) : 1.f;
        bl[i] = ok ? __ldg(p.bh + (size_t)ge * D::Nq + l) : 0.f;
        if (EARLY) load_rk(i);
    }
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, parity, p.status))) return false;
    parity ^= 1;
    __syncwarp();
    // ---- flux differencing over all columns, rows l = b + LPE*i ------------------
    const float4* utE = reinterpret_cast<const float4*>(ws + C::w_ut + e * C::UTS);
    const float4* geE = reinterpret_cast<const float4*>(ws + C::w_geo + e * C::UTS);
    // the free surface relative to the element's first node in the pressure
    // and bathymetry terms: exact by Q_SBP 1 = 0 (Theorem 3.1), and the FP32
    // sums no longer cancel large equal terms (as in k_stage2)
    const float Href = utE[0].w;
    float rh[RPL], ru[RPL], rv[RPL], rrx[RPL], rsx[RPL], rry[RPL], rsy[RPL];
    float a0[RPL], a1[RPL], a2[RPL];
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int l = b + LPE * i;
        float4 U = make_float4(1.f, 0.f, 0.f, 1.f), G = make_float4(0.f, 0.f, 0.f, 0.f);
        if (l < D::Nq) {
            U = utE[l];
            G = geE[l];
        }
        rh[i] = U.x;
        ru[i] = U.y;
        rv[i] = U.z;
        rrx[i] = G.x;
        rsx[i] = G.y;
        rry[i] = G.z;
        rsy[i] = G.w;
        a0[i] = a1[i] = a2[i] = 0.f;
    }
    const float* QsB = ops + C::o_Qs + b * C::OPB;
#define ESDG_SBP_PAIR(I, QR, QS)                                               \
{                                                                          \
    const float Qx = (QR) * (rrx[I] + G.x) + (QS) * (rsx[I] + G.y);        \
    const float Qy = (QR) * (rry[I] + G.z) + (QS) * (rsy[I] + G.w);        \
    const float HU = fmaf(rh[I], ru[I], hum), HV = fmaf(rh[I], rv[I], hvm);\
    const float T = fmaf(Qx, HU, Qy * HV);                                 \
    const float P = rh[I] * gH2;                                           \
    a0[I] += T;                                                            \
    a1[I] = fmaf(U.y, T, fmaf(Qx, P, a1[I]));                              \
    a2[I] = fmaf(U.z, T, fmaf(Qy, P, a2[I]));                              \
}
#pragma unroll 2
    for (int m = 0; m < D::Nq; ++m) {
        const float4 U = utE[m], G = geE[m];
        const float hum = U.x * U.y, hvm = U.x * U.z, gH2 = 2.f * g * (U.w - Href);
        const float4* q4 = reinterpret_cast<const float4*>(QsB + m * LPE * C::OPB);
#pragma unroll
        for (int i2 = 0; i2 < (RPL + 1) / 2; ++i2) {
            const float4 q = q4[i2];
            ESDG_SBP_PAIR(2 * i2, q.x, q.y)
            if (2 * i2 + 1 < RPL) ESDG_SBP_PAIR(2 * i2 + 1, q.z, q.w)
        }
    }
#undef ESDG_SBP_PAIR
    int bad = 0;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int l = b + LPE * i;
        a1[i] = fmaf(ru[i], a0[i], a1[i]);
        a2[i] = fmaf(rv[i], a0[i], a2[i]);
        a0[i] *= 2.f;
        if (l >= D::Nq) continue;
        // ---- interface flux at a face node (well-balanced pressure, LF) -----------
        const int f = frow[l];
        if (f >= 0) {
            const float4 tp = *reinterpret_cast<const float4*>(ws + C::w_tr + (e * D::Nfq + f) * 4);
            const float h_l = rh[i];
            const float nr = ops[C::o_nrs + 2 * f], ns = ops[C::o_nrs + 2 * f + 1];
            const float nxJ = rrx[i] * nr + rsx[i] * ns;
            const float nyJ = rry[i] * nr + rsy[i] * ns;
            const float hP = tp.x, uP = tp.y, vP = tp.z;
            const float huP = hP * uP, hvP = hP * vP;
            const float w = ops[C::o_wf + f];
            const float hu_l = h_l * ru[i], hv_l = h_l * rv[i];
            const float huA = 0.5f * (hu_l + huP), hvA = 0.5f * (hv_l + hvP);
            const float uA = 0.5f * (ru[i] + uP), vA = 0.5f * (rv[i] + vP);
            const float pw = 0.5f * g * h_l * ((hP - h_l) + (utE[l].w - Href));  // (h+ + b_l) - Href
            const float Fn0 = nxJ * huA + nyJ * hvA;
            a0[i] += w * Fn0;
            a1[i] += w * (uA * Fn0 + nxJ * pw);
            a2[i] += w * (vA * Fn0 + nyJ * pw);
            if (p.lf) {
                // sJ max(|u.n| + sqrt(g h)) over both sides, with the unit normal
                // n = nJ / sJ folded in: |u.nJ| + sqrt(sJ^2 g h) (no divisions)
                const float sJ2 = nxJ * nxJ + nyJ * nyJ;
                const float lm = fabsf(ru[i] * nxJ + rv[i] * nyJ) + sqrtf(sJ2 * g * h_l);
                const float lp = fabsf(uP * nxJ + vP * nyJ) + sqrtf(sJ2 * g * hP);
                const float c = 0.5f * w * fmaxf(lm, lp);
                a0[i] -= c * (hP - h_l);
                a1[i] -= c * (huP - hu_l);
                a2[i] -= c * (hvP - hv_l);
            }
        }
        // ---- du/dt = -r / (w J) + forcing -------------------------------------------
        const float iw = 1.f / wj[i];
        float d[3] = {-a0[i] * iw, -a1[i] * iw, -a2[i] * iw};
        if (p.forcing && valid) {
            const float x = p.xq[(size_t)ge * D::Nq + l], y = p.yq[(size_t)ge * D::Nq + l];
            float sth, cth, sx, cx, sy, cy;
            sincospif(x + y - (float)p.t, &sth, &cth);
            sincospif(x, &sx, &cx);
            sincospif(y, &sy, &cy);
            const float pi = 3.14159265358979323846f;
            const float h = 2.f + p.mms_amp * sth;
            const float cc = p.mms_amp * pi * cth;
            const float bx = -p.mms_bamp * pi * sx * cy, by = -p.mms_bamp * pi * cx * sy;
            const float u0 = p.mms_u0, v0 = p.mms_v0;
            d[0] += -cc + u0 * cc + v0 * cc;
            d[1] += -u0 * cc + (u0 * u0 + g * h) * cc + u0 * v0 * cc + g * h * bx;
            d[2] += -v0 * cc + u0 * v0 * cc + (v0 * v0 + g * h) * cc + g * h * by;
        }
        if (!valid) continue;
        if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) p.rhs_out[((size_t)c * K + ge) * D::Nq + l] = (double)d[c];
        } else {
            // ---- LSRK45 stage in FP64; the next stage's record --------------------------
            // (dt du/dt formed in FP32, the precision of du/dt; the record's
            // velocities divided in FP32, the precision they are stored in: the
            // FP64 pipe, narrow on this part, keeps only the two DFMAs a value)
            if (!EARLY) load_rk(i);
            const float dtf = (float)p.dt;
            float uf[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const size_t gi = ((size_t)c * K + ge) * D::Nq + l;
                const double rs = fma(p.rkA, ro[i][c], f2d_bits(dtf * d[c]));
                const double un = fma(p.rkB, rs, uo[i][c]);
                p.res[gi] = rs;
                p.u[gi] = un;
                if (p.u_out) p.u_out[gi] = un;
                uf[c] = d2f_bits(un);
            }
            if (!(uf[0] > 0.f)) bad |= STATUS_NONPOSITIVE;
            if (!isfinite(uf[0]) || !isfinite(uf[1]) || !isfinite(uf[2])) bad |= STATUS_NONFINITE;
            const float ih = 1.f / uf[0];
            *reinterpret_cast<float4*>(p.ut_out + ((size_t)ge * D::Nq + l) * 4) =
                make_float4(uf[0], uf[1] * ih, uf[2] * ih, uf[0] + bl[i]);
        }
    }
    if (bad) atomicOr(p.status, bad);
    // reads of the staging area are done before the next batch's bulk copies
    fence_proxy_async_smem();
    __syncwarp();
    return true;
}

// MODE 0: du/dt into rhs_out; MODE 1: LSRK45 stage and the next records.
template <int N, int MODE>
__global__ void __launch_bounds__(S2<N>::WARPS * 32, 1) k_sbp2(StageParams<float> p, const float* __restrict__ ops2,
                                                               int Kpad) {
    typedef S2<N> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* ops = reinterpret_cast<float*>(smem_raw);
    const int nwarps = blockDim.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ops + C::o_end + nwarps * C::w_end);
    for (int i = threadIdx.x; i < C::o_end / 4; i += blockDim.x)
        reinterpret_cast<float4*>(ops)[i] = reinterpret_cast<const float4*>(ops2)[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) mbar_init(&bars[warp], 1);
    fence_mbar_init();
    __syncthreads();
    uint64_t* bar = &bars[warp];
    float* ws = ops + C::o_end + warp * C::w_end;
    uint32_t parity = 0;
    const int nbatch = Kpad / C::EPW;
    for (int batch = blockIdx.x * nwarps + warp; batch < nbatch; batch += gridDim.x * nwarps)
        if (!sbp2_batch<N, MODE>(p, ops, ws, bar, parity, batch * C::EPW, lane)) return;
}

}  // namespace esdg
