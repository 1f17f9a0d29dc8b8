// Batched FP32 stage kernel for sm_103a (RHS in FP32, RK state in FP64).
//
// Same operator as k_stage (the split form of Sec. 5.2 with the curved metric
// average of Sec. 2.7, the EC flux of eqs. (SWE_flux1/2) with its folded
// well-balanced bathymetry term, interface flux + Lax-Friedrichs of Sec. 2.8,
// lift, stored inverse curved mass matrix, LSRK45 stage of Sec. 4, and the
// entropy projection of Sec. 2.6 for the next stage), mapped differently:
//
//  * a warp processes a batch of EPW = 32/LPE = 4 elements; LPE = 8 lanes share
//    one element.  Lane (e, b) owns the hybrid rows l = b + LPE*i, i < RPL,
//    with their node data and three accumulators in registers, so a column m
//    is read from shared memory once for RPL rows (the flux differencing is
//    FP32-ALU bound, and this keeps shared-memory traffic well below it).
//    Eight lanes per element (rather than four) halve the registers and the
//    shared memory per warp, which lets 24 warps share an SM.
//    Interleaving rows across the LPE lanes balances volume rows (all Nh
//    columns) against face rows (Nq columns: the lower-right block of
//    Q_skew is zero).
//  * the element data of a batch (u~, metrics, inverse mass) arrive in
//    shared memory by TMA bulk copies (cp.async.bulk) on a per-warp mbarrier,
//    one copy per element into slots padded so that the column reads of the
//    EPW elements of a warp fall in distinct banks.  The wait is bounded.
//  * lift, inverse mass and projection spread modes, nodes or fields over
//    the LPE lanes of an element, with the permuted operators in shared
//    memory laid out so each lane reads contiguous float4s.
//  * with the weight-adjusted inverse mass (Dims::wadg; Sec. 2.8 names it as
//    the way to avoid stored inverses) no per-element matrix is stored or
//    copied: the inverse Vq^T diag(w/J) Vq is applied through shared factors
//    composed on the host (C = Vq Vh^T, A = Vq Vq^T, B = Vh Vq^T) and a
//    per-node scale w^2 / (w J).
#pragma once

#include "esdg_kernels.cuh"
#include "esdg_tc.cuh"

namespace esdg {

constexpr int STATUS_TIMEOUT = 4;

template <int N>
struct C2 {
    typedef Dims<N> D;
    static constexpr int LPE = 8;                           // lanes per element
    static constexpr int EPW = 32 / LPE;                    // elements per warp
    static constexpr int RPL = (D::Nh + LPE - 1) / LPE;     // hybrid rows per lane
    static constexpr int QPL = (D::Nq + LPE - 1) / LPE;     // volume nodes per lane
    static constexpr int MPL = (D::Np + LPE - 1) / LPE;     // modes per lane
    // operator entries per (column, lane slot): a multiple of 4 with an odd
    // quotient, so the 8 lanes' float4 reads of one column hit 8 distinct
    // 4-bank groups
    static constexpr int OPB = ((2 * RPL + 3) / 4) % 2 == 1 ? (2 * RPL + 3) / 4 * 4 : (2 * RPL + 3) / 4 * 4 + 4;
    static constexpr int RPLp = (RPL + 3) & ~3;
    static constexpr int QPLp = (QPL + 3) & ~3;
    static constexpr int MPLp = (MPL + 3) & ~3;
    static constexpr int NpP4 = (D::NpP + 3) & ~3;          // padded packed inverse-mass stride
    // element slot of u~ / metric staging: the EPW elements' float4 records of
    // one node fall in distinct 4-bank groups (slot stride not 0 or 16 mod 32)
    static constexpr int UTS = ((D::Nh * 4 + 4) % 32 == 0 || (D::Nh * 4 + 4) % 32 == 16) ? D::Nh * 4 + 8 : D::Nh * 4 + 4;
    static constexpr int MIS = NpP4 + 4;                    // element slot of inverse-mass staging
    static constexpr bool WADG = D::wadg;                   // weight-adjusted inverse mass
    // Dense contractions on the tensor cores (stored inverse only): per warp,
    // the rows (element e, field f) -> 3 e + f of an M = 64 TF32 MMA whose
    // other 48 rows are never read, N = 16 columns of TMEM per warp.
    static constexpr bool TC = D::tc;
    static_assert(!(TC && WADG), "tensor-core path: stored inverse only");
    static constexpr int TN = 16;                                   // MMA N, TMEM columns per warp
    static constexpr int KL = (D::Nh + 7) & ~7;                     // K of the lift (hybrid nodes)
    static constexpr int KM = (D::Np + 7) & ~7;                     // K over modes
    static constexpr int KQ = (D::Nq + 7) & ~7;                     // K over volume nodes
    static constexpr int KA = KL > KM ? (KL > KQ ? KL : KQ) : (KM > KQ ? KM : KQ);
    static constexpr int NpR = (D::Np + 15) & ~15, NqR = (D::Nq + 15) & ~15, NhR = (D::Nh + 15) & ~15;
    // B operand blocks in the operator region (floats; hi part, then lo part
    // at + rows * K): lift Vh^T (rows modes, K hybrid nodes), Vq (rows volume
    // nodes, K modes), Vq^T (rows modes, K volume nodes), Vh (rows hybrid
    // nodes, K modes)
    static constexpr int tb_lift = 0;
    static constexpr int tb_vq = tb_lift + 2 * NpR * KL;
    static constexpr int tb_vqt = tb_vq + 2 * NqR * KM;
    static constexpr int tb_vh = tb_vqt + 2 * NpR * KQ;
    static constexpr int tb_end = tb_vh + 2 * NhR * KM;
    // operator region (floats).  Stored inverse: lift Vh^T, projection Vq^T,
    // interpolation Vq and Vh.  Weight-adjusted inverse Vq^T diag(w/J) Vq
    // with the shared factors composed: C = Vq Vh^T (lift to the volume
    // nodes), A = Vq Vq^T, B = Vh Vq^T, so that
    //   du/dt = -Vq^T [(w/J) o (C r - A (w J f))]   and
    //   v~    =  B [(w/J) o (A (w J v))].
    static constexpr int o_Qs = 0;                                  // [Nh][LPE][OPB]
    // Unique pairs (UP; volume rules of 2 LPE points, so that slots i < VS of
    // every lane hold volume rows and the slots above face rows): each
    // non-zero pair of Q_skew is evaluated once, by the lane of its volume
    // row l = b + LPE i, against a partner row m = c + LPE j of lane c = (b + s)
    // mod LPE at offset s; row m's share (Q_skew is skew and the flux
    // symmetric) reaches lane c by a shuffle.  Volume-volume pairs: offset 0
    // (rows b and b + LPE of one lane) and offsets 1..LPE/2 (at LPE/2 each
    // lane pair splits its four pairs two and two); volume-face pairs: offsets
    // 0..LPE-1.  Tables of (Qr, Qs) entries in that order, zero where a pair
    // is not this lane's or m is past Nh:
    //   o_U0  [LPE][2]               pair (b, b + LPE)
    //   o_Uvv [LPE/2][VS][LPE][4]    (l0, m), (l1, m) at offset s = 1.., slot j
    //   o_Uvf [LPE][FS][LPE][4]      the same at offset s = 0.., face slot VS + j
    static constexpr int VS = D::Nq / LPE;                  // volume row slots
    static constexpr int FS = RPL - VS;                     // face row slots
#ifndef ESDG_STAGE2_UNIQUE_PAIRS
#define ESDG_STAGE2_UNIQUE_PAIRS 1
#endif
    static constexpr bool UP = ESDG_STAGE2_UNIQUE_PAIRS && D::Nq == 2 * LPE;
    static constexpr int o_U0 = o_Qs;
    static constexpr int o_Uvv = o_U0 + 2 * LPE;
    static constexpr int o_Uvf = o_Uvv + (LPE / 2) * VS * LPE * 4;
    static constexpr int QS_FLOATS = UP ? o_Uvf + LPE * FS * LPE * 4 : D::Nh * LPE * OPB;
    static constexpr int o_VhT = o_Qs + QS_FLOATS;                  // [Nh][LPE][MPLp]: Vh[l][b+LPE j]
    static constexpr int o_tc = o_VhT;                              // tensor-core B blocks (TC)
    static constexpr int o_VqT = o_VhT + (TC ? tb_end : WADG ? 0 : D::Nh * LPE * MPLp);  // [Nq][LPE][MPLp]: Vq[q][b+LPE j]
    static constexpr int o_Vq = o_VqT + (TC ? 0 : D::Nq * LPE * MPLp);      // [Np][LPE][QPLp]: Vq[b+LPE j][n]
    static constexpr int o_Vh = o_Vq + (TC ? 0 : D::Np * LPE * QPLp);       // [Np][LPE][RPLp]: Vh[b+LPE j][n]
    static constexpr int o_C = o_Vh + ((WADG || TC) ? 0 : D::Np * LPE * RPLp);  // [Nh][LPE][QPLp]: C[b+LPE j][l]
    static constexpr int o_A = o_C + (WADG ? D::Nh * LPE * QPLp : 0);      // [Nq][LPE][QPLp]: A[b+LPE j][q]
    static constexpr int o_B = o_A + (WADG ? D::Nq * LPE * QPLp : 0);      // [Nq][LPE][RPLp]: B[b+LPE j][q]
    static constexpr int o_wq = o_B + (WADG ? D::Nq * LPE * RPLp : 0);     // [Nq] volume weights
    static constexpr int o_wf = o_wq + (WADG ? D::Nq : 0);          // [Nfq]
    static constexpr int o_nrs = o_wf + D::Nfq;                     // [Nfq][2]
    static constexpr int o_end = (o_nrs + 2 * D::Nfq + 3) & ~3;
    // per-warp region (floats)
    static constexpr int w_ut = 0;                          // [EPW][UTS]  h u v H
    static constexpr int w_geo = w_ut + EPW * UTS;          // [EPW][UTS]  rxJ sxJ ryJ syJ (scaled 1/8)
    static constexpr int w_tr = w_geo + EPW * UTS;          // [EPW][Nfq][4] neighbour traces
    // tensor-core scratch (TC) sizes, laid out below
    static constexpr int KMQ = KM > KQ ? KM : KQ;
    static constexpr int TES = 72, TFS = 20;                 // t_in: element and field strides
    static constexpr int VES = 3 * NhR + 24, VFS = NhR + 8;  // t_vt: element and field strides
    static constexpr int t_in_ = 32 * KMQ;
    static constexpr int t_end_ = t_in_ + ((EPW - 1) * TES + 3 * TFS > (EPW - 1) * VES + 3 * VFS
                                               ? (EPW - 1) * TES + 3 * TFS
                                               : (EPW - 1) * VES + 3 * VFS);
    static constexpr int w_mi0 = w_tr + EPW * D::Nfq * 4;
    // the M = 64 products read A rows of the neighbouring quarters: up to
    // 32 KA + 192 floats past the operand for the warp of quarter 0, kept
    // inside the warp's region
    static constexpr int t_read_ = 32 * KA + 192;
    static constexpr int t_need_ = t_end_ > t_read_ ? t_end_ : t_read_;
    static constexpr int w_mi = (TC && t_need_ > w_mi0) ? (t_need_ + 3) & ~3 : w_mi0;  // [EPW][MIS]  packed (M_h^k)^-1
    static constexpr int w_end = (w_mi + (WADG ? 0 : EPW * MIS) + 3) & ~3;
    // scratch aliases, live after the volume/interface phase
    static constexpr int s_rt = w_ut;                       // [3][Nh][EPW]
    static constexpr int s_t = w_geo;                       // [3][Nq][EPW]
    static constexpr int s_s = w_geo + 3 * D::Nq * EPW;     // [3][Np][EPW]
    static constexpr int s_u = w_tr;                        // [3][Np][EPW]
    static_assert(3 * D::Nh <= UTS, "rt scratch");
    static_assert(3 * D::Nq * EPW + 3 * D::Np * EPW <= EPW * UTS, "t/s scratch");
    static_assert(3 * D::Np <= D::Nfq * 4, "u scratch");
    // tensor-core scratch (TC), aliasing the staging after the volume phase:
    // t_A the A operand of a contraction over K (16 rows x K, the hi part,
    // then the lo part at + 16 K; row r, column k at (k / 4) 64 + (r / 8) 32 +
    // (r % 8) 4 + k % 4: K-direction core matrices 256 bytes apart, 8-row
    // groups 128 bytes apart); t_in the 16-column MMA results of row (e, f)
    // at e TES + f TFS, past the operands over modes and volume nodes; t_vt
    // the values at the hybrid nodes, row (e, f) at e VES + f VFS, in the same
    // place (t_in is consumed by then).  Strides chosen so that the readers
    // (8 lanes of each of the 4 elements) hit distinct banks.
    static constexpr int t_A = 0;
    static constexpr int t_in = t_in_;
    static constexpr int t_vt = t_in_;
    static_assert(!TC || (D::Np <= 16 && D::Nq <= 16), "tensor-core path: one 16-column round for Vq, Vq^T, lift");
    static_assert(!TC || TFS >= 16 && VFS >= NhR, "row strides");
    static_assert(!TC || t_end_ <= w_mi, "tensor-core scratch below the inverse-mass staging");
    // the M = 64 products read A rows of the neighbouring quarters: up to the
    // lo part's end plus 6 row groups for the warp of quarter 0, which must
    // stay inside the warp's region
    static_assert(!TC || 64 * KA + (KA / 4 - 1) * 256 + 8 * 128 <= 4 * w_end, "A operand reads inside the region");
    static constexpr int TRL = (EPW * D::Nfq + 31) / 32;    // neighbour traces gathered per lane
    static constexpr int RKL = (3 * EPW * D::Np + 31) / 32; // RK values per lane (all 32 lanes)
    // the RK update at the modes n = b + LPE j whose du/dt the inverse mass
    // leaves in a lane's registers, where that takes no more FP64 warp
    // instructions than spreading the batch's values over all 32 lanes
    // (N = 2, 4; measured 2-5% faster there, 4% slower at N = 3)
    static constexpr bool RK_LANES = 3 * MPL <= RKL;
    // RK operands loaded before the lift, else just before the update: late
    // only for the 31 hybrid nodes of N = 4 with the 16-point rule and the
    // stored inverse, where the early loads push the kernel past 80
    // registers (measured per configuration; elsewhere early is faster)
    static constexpr bool EARLY_RK = !(D::Nh == 31 && D::Nq == 16 && !WADG);
    // column unroll of the volume loops: 1 for the 31 hybrid nodes of N = 4
    // with the 16-point rule (178.0 against 180.8 us per stage at K = 131072),
    // 2 elsewhere (N = 3 and the collapsed rules ran 0.6-1.2% faster with 2)
    static constexpr int VUNROLL = (D::Nh == 31 && D::Nq == 16) ? 1 : 2;
    // warps per CTA (one CTA per SM): as many as fit in 227 KB of shared
    // memory next to the operators, at most 24 (80 registers per thread) for
    // volume rules of up to 16 points and 16 (128 registers) above, where the
    // row and node data no longer fit 80 registers without spilling.  More
    // resident warps hide more of the latency this issue-bound kernel waits on:
    // 24 warps at 80 registers ran 5% (N = 4) to 11% (N = 3) faster than 16 at
    // 128; 28 at 72 registers spilled and ran slower.
    static constexpr int SMEM_MAX = 232448;
    static constexpr int WARPS_FIT = (SMEM_MAX - 4 * o_end) / (4 * w_end + 8);
    static constexpr int WARPS_CAP = D::Nq <= 16 ? 24 : 16;
    static constexpr int WARPS = WARPS_FIT < WARPS_CAP ? WARPS_FIT : WARPS_CAP;
    // per-warp mbarriers of the bulk copies; TC: per-warp MMA-completion
    // mbarriers (byte offset tc_bar), the TMEM address (tc_slot) and the
    // per-warp phases of the MMA barriers (tc_par)
    static constexpr int tc_bar = 4 * (o_end + WARPS * w_end) + 8 * WARPS;
    static constexpr int tc_slot = tc_bar + 8 * WARPS;
    static constexpr int tc_par = tc_slot + 16;
    static constexpr size_t bytes() {
        return sizeof(float) * (size_t(o_end) + size_t(WARPS) * w_end) + 8 * WARPS + (TC ? 8 * WARPS + 16 + 4 * WARPS : 0);
    }
    static constexpr int TX_BYTES = EPW * (2 * D::Nh * 16 + (WADG ? 0 : NpP4 * 4));
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Wait for phase `parity` of bar, giving up after ~2^31 SM cycles (about a
// second): then the status word gets STATUS_TIMEOUT and the caller returns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) {
            atomicOr(status, STATUS_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Exact float -> double and round-to-nearest-even double -> float conversions
// done on the integer pipes (the FP64 pipe, where the conversion instructions
// run, is narrow on this part); zeros and normal numbers take the bit path,
// everything else (subnormals, infinities, NaN, out-of-range) the built-in
// conversion.
__device__ __forceinline__ double f2d_bits(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t ex = (b >> 23) & 0xffu;
    if (ex - 1u < 254u) {
        const uint32_t man = b & 0x7fffffu;
        return __hiloint2double((int)((b & 0x80000000u) | ((ex + 896u) << 20) | (man >> 3)), (int)(man << 29));
    }
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
    return (double)x;
}
__device__ __forceinline__ float d2f_bits(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t ex = (hi >> 20) & 0x7ffu;
    if (ex - 897u < 254u) {
        const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const uint32_t rest = lo & 0x1fffffffu;
        uint32_t f = (hi & 0x80000000u) | ((ex - 896u) << 23) | m;
        f += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
        return __uint_as_float(f);
    }
    if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(hi & 0x80000000u);
    return (float)d;
}

// Rows n = b + LPE j of (M_h^k)^{-1} y for the three fields; y[f][m] at
// y + f * YF + m * YM (default: [field][mode][element]); M the packed lower
// triangle.
template <int Np, int MPL, int LPE, int EPW, int YF = Np * EPW, int YM = EPW>
__device__ __forceinline__ void minv_rows(const float* __restrict__ M, const float* y, int b, float (&r0)[MPL],
                                          float (&r1)[MPL], float (&r2)[MPL]) {
    const float* rowp[MPL];
    const float* colp[MPL];
#pragma unroll
    for (int j = 0; j < MPL; ++j) {
        const int n = b + LPE * j;
        rowp[j] = M + n * (n + 1) / 2;  // M[n][m] = rowp[m] for m <= n
        colp[j] = M + n;                 // M[n][m] = colp[m (m + 1) / 2] for m > n
        r0[j] = r1[j] = r2[j] = 0.f;
    }
#pragma unroll
    for (int m = 0; m < Np; ++m) {
        const float y0 = y[m * YM], y1 = y[YF + m * YM], y2 = y[2 * YF + m * YM];
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const int n = b + LPE * j;
            if (n < Np) {
                const float mv = m <= n ? rowp[j][m] : colp[j][m * (m + 1) / 2];
                r0[j] = fmaf(mv, y0, r0[j]);
                r1[j] = fmaf(mv, y1, r1[j]);
                r2[j] = fmaf(mv, y2, r2[j]);
            }
        }
    }
}

// ---- tensor-core rounds (TC) ---------------------------------------------------
// Offset in an A operand of row r and column k = b + 8 j is tc_off(r, b) +
// 128 j (columns b + 8 j of a lane b of the 8 lanes of an element).
__device__ __forceinline__ int tc_off(int r, int b) { return (b >> 2) * 64 + (b & 3) + (r >> 3) * 32 + (r & 7) * 4; }

// The TF32 pair (hi, lo) of v at offset o of an A operand with K columns.
__device__ __forceinline__ void tc_put_at(float* A, int K, int o, float v) {
    const float hi = tf32_rn(v);
    A[o] = hi;
    A[16 * K + o] = tf32_rn(v - hi);
}

// The same at row r, any column k.
__device__ __forceinline__ void tc_put(float* A, int K, int r, int k, float v) {
    tc_put_at(A, K, tc_off(r, k & 7) + 128 * (k >> 3), v);
}

// Lanes i < 3 EPW: row i = (element i / 3, field i % 3) of an MMA result,
// 16 values, to dst + e es + f fs.
template <int EPW>
__device__ __forceinline__ void tc_store_rows(float* dst, int es, int fs, int lane, const float (&d)[16]) {
    if (lane < 3 * EPW) {
        const int re = lane / 3, rf = lane - (lane / 3) * 3;
        float4* o = reinterpret_cast<float4*>(dst + re * es + rf * fs);
#pragma unroll
        for (int i = 0; i < 4; ++i) o[i] = make_float4(d[4 * i], d[4 * i + 1], d[4 * i + 2], d[4 * i + 3]);
    }
}

// try_wait with a suspend-time hint: the thread sleeps until the phase
// completes or about the hinted time passes, instead of spinning
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

// The warp's MMA-completion barrier and its state word (bit 0: the phase to
// wait for; bit 1: a wait expired, after which the warp issues no more MMAs).
template <int NR>
__device__ __forceinline__ uint64_t* tc_bar_of_warp() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<uint64_t*>(smem_raw + C2<NR>::tc_bar) + (threadIdx.x >> 5);
}
template <int NR>
__device__ __forceinline__ uint32_t* tc_state_of_warp() {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return reinterpret_cast<uint32_t*>(smem_raw + C2<NR>::tc_par) + (threadIdx.x >> 5);
}

// D = A B^T over K (A: this warp's 16 rows at A, K columns; B: 16 rows of a
// B block, hi part at Bhi and lo part at Blo, row n, column k at (n / 8) 8 K +
// (k / 4) 32 + (n % 8) 4 + k % 4), accumulated onto the previous round's D
// when acc0; then, with LOAD, thread i < 16 gets row i of D (16 columns).
// Three TF32 products per K step of 8 (hi hi, lo hi, hi lo).  The A
// descriptor starts 16 q rows before this warp's rows (q = warp mod 4), so
// that they are rows 16 q .. 16 q + 15 of the M = 64 product and land in the
// warp's own TMEM lane quarter; the other 48 rows read whatever shared memory
// lies there (inside the block's allocation) and their results are never
// read.  The warp's TMEM columns, MMA barrier and state word sit at fixed
// places of the block's shared memory (C::tc_slot, C::tc_bar, C::tc_par).
// If the bounded wait for the MMAs expires, status gets STATUS_TIMEOUT, the
// warp's state records it, and this and later rounds of the warp do nothing
// (the batch loop then stops; the results of the batch are not used).
template <int NR, int K, bool LOAD = true>
__device__ __forceinline__ void tc_round(const float* A, const float* Bhi, const float* Blo, bool acc0, int* status,
                                         int lane, float (&v)[16]) {
    typedef C2<NR> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int w = threadIdx.x >> 5, q = w & 3;
    uint64_t* bar = tc_bar_of_warp<NR>();
    uint32_t* st = tc_state_of_warp<NR>();
    const uint32_t tbase = *reinterpret_cast<const uint32_t*>(smem_raw + C::tc_slot) + (uint32_t)(C::TN * w);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes of A -> tensor-core reads
    __syncwarp();
    const uint32_t s0 = *st;
    if (s0 & 2u) return;
    if (lane == 0) {
        tc_fence_after();
        // descriptors of the first K step; a step of 8 advances A by two
        // K-direction core matrices (512 bytes) and B by two (256 bytes), i.e.
        // the start-address field (bytes / 16) by 32 and 16
        const uint32_t a0 = smem_u32(A) - 256u * (uint32_t)q;
        const uint64_t ahi = tc_sdesc(a0, 256u, 128u), alo = tc_sdesc(a0 + 64u * K, 256u, 128u);
        const uint64_t bhi = tc_sdesc(smem_u32(Bhi), 128u, 32u * K), blo = tc_sdesc(smem_u32(Blo), 128u, 32u * K);
        constexpr uint32_t id = tc_idesc_tf32(64, 16);
#pragma unroll
        for (int kc = 0; kc < K / 8; ++kc) {
            tc_mma_tf32(tbase, ahi + 32u * kc, bhi + 16u * kc, id, (acc0 || kc > 0) ? 1u : 0u);
            tc_mma_tf32(tbase, alo + 32u * kc, bhi + 16u * kc, id, 1u);
            tc_mma_tf32(tbase, ahi + 32u * kc, blo + 16u * kc, id, 1u);
        }
        tc_commit(smem_u32(bar));
    }
    const uint32_t ph = s0 & 1u;
    const long long t0 = clock64();
    bool ok = true;
    while (!mbar_try_wait_sleep(bar, ph)) {
        if (clock64() - t0 > (1LL << 31)) {
            ok = false;
            break;
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();  // every lane has read the state word
    if (lane == 0) {
        if (ok) {
            *st = ph ^ 1u;
        } else {
            *st = s0 | 2u;
            atomicOr(status, STATUS_TIMEOUT);
        }
    }
    __syncwarp();
    if (!ok) return;
    tc_fence_after();
    if constexpr (LOAD) tc_ld16(tbase + ((uint32_t)(32 * q) << 16), v);
    tc_fence_before();
}

// true once one of the warp's MMA waits has expired
template <int NR>
__device__ __forceinline__ bool tc_failed() {
    return (*tc_state_of_warp<NR>() & 2u) != 0;
}

// Neighbour traces of the batch starting at e0 (a gather): lane handles
// k = lane + 32 t, element k / Nfq, face node k % Nfq.
template <int N>
__device__ __forceinline__ void gather_traces(const StageParams<float>& p, const float* __restrict__ ut_in, int e0,
                                              int lane, float4 (&tv)[C2<N>::TRL]) {
    typedef Dims<N> D;
#pragma unroll
    for (int t = 0; t < C2<N>::TRL; ++t) {
        const int k = lane + 32 * t;
        tv[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < C2<N>::EPW * D::Nfq) {
            const int ee = k / D::Nfq, f = k - ee * D::Nfq;
            const int face = f / D::Nfp, i = f - face * D::Nfp;
            const int nb = __ldg(p.nbr + (size_t)(e0 + ee) * 3 + face);
            const int en = nb >> 2, fn = nb & 3;
            if (fn != 3)  // 3: a wall, whose exterior state is built from the own trace
                tv[t] = __ldg(reinterpret_cast<const float4*>(
                    ut_in + ((size_t)en * D::Nh + D::Nq + fn * D::Nfp + (D::Nfp - 1 - i)) * 4));
        }
    }
}

// The projection chain of stage2_project on the tensor cores: the new FP32
// state u is already in the A operand (rows 3 e + f, K over modes).
// u_q = Vq u (MMA), v(u_q) w J at this lane's volume nodes, y = Vq^T (w J v)
// (MMA), v_h = (M_h^k)^{-1} y (per element, FP32 pipes), v~ = Vh v_h (MMA, in
// 16-node chunks) into v0..v2 at the lane's hybrid rows.
template <int N>
__device__ __forceinline__ void tc_project(const StageParams<float>& p, const float* __restrict__ ops, const float* Mi,
                                           float* ws, int ge, int lane, const float (&bqv)[C2<N>::QPL],
                                           const float (&wqv)[C2<N>::QPL], float (&v0)[C2<N>::RPL],
                                           float (&v1)[C2<N>::RPL], float (&v2)[C2<N>::RPL], int& bad) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL, QPL = C::QPL, MPL = C::MPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const float g = p.g;
    const bool valid = ge < p.K;
    float* tA = ws + C::t_A;
    float* tin = ws + C::t_in;
    const float* tb = ops + C::o_tc;
    int of[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) of[f] = tc_off(3 * e + f, b);
    float d[16] = {};
    // u_q = Vq u
    tc_round<N, C::KM>(tA, tb + C::tb_vq, tb + C::tb_vq + C::NqR * C::KM, false, p.status, lane, d);
    tc_store_rows<EPW>(tin, C::TES, C::TFS, lane, d);
    __syncwarp();
    // w J v(u_q) at q = b + LPE j into the A operand over the volume nodes
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = b + LPE * j;
        if (q < C::KQ) {
            float t0 = 0.f, t1 = 0.f, t2 = 0.f;
            if (valid && q < D::Nq) {
                const float* u = tin + e * C::TES + q;
                const float h = u[0];
                if (!(h > 0.f)) bad |= STATUS_NONPOSITIVE;
                const float ih = 1.f / h;
                const float uu = u[C::TFS] * ih, vv = u[2 * C::TFS] * ih;
                const float wj = wqv[j];
                t0 = wj * (g * (h + bqv[j]) - 0.5f * (uu * uu + vv * vv));
                t1 = wj * uu;
                t2 = wj * vv;
            }
            tc_put_at(tA, C::KQ, of[0] + 128 * j, t0);
            tc_put_at(tA, C::KQ, of[1] + 128 * j, t1);
            tc_put_at(tA, C::KQ, of[2] + 128 * j, t2);
        }
    }
    // y = Vq^T (w J v)
    tc_round<N, C::KQ>(tA, tb + C::tb_vqt, tb + C::tb_vqt + C::NpR * C::KQ, false, p.status, lane, d);
    tc_store_rows<EPW>(tin, C::TES, C::TFS, lane, d);
    __syncwarp();
    // v_h = (M_h^k)^{-1} y into the A operand over the modes (zero past Np)
    {
        float r0[MPL], r1[MPL], r2[MPL];
        minv_rows<D::Np, MPL, LPE, EPW, C::TFS, 1>(Mi, tin + e * C::TES, b, r0, r1, r2);
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const bool in = b + LPE * j < D::Np;
            tc_put_at(tA, C::KM, of[0] + 128 * j, in ? r0[j] : 0.f);
            tc_put_at(tA, C::KM, of[1] + 128 * j, in ? r1[j] : 0.f);
            tc_put_at(tA, C::KM, of[2] + 128 * j, in ? r2[j] : 0.f);
        }
    }
    // v~ = Vh v_h, 16 hybrid nodes a round (t_vt aliases t_in, consumed by now)
    float* tvt = ws + C::t_vt;
#pragma unroll 1
    for (int c = 0; c < C::NhR / 16; ++c) {
        tc_round<N, C::KM>(tA, tb + C::tb_vh + 16 * C::KM * c, tb + C::tb_vh + (C::NhR + 16 * c) * C::KM, false,
                    p.status, lane, d);
        tc_store_rows<EPW>(tvt + 16 * c, C::VES, C::VFS, lane, d);
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int l = b + LPE * j;
        const float* v = tvt + e * C::VES + (l < D::Nh ? l : 0);
        v0[j] = v[0];
        v1[j] = v[C::VFS];
        v2[j] = v[2 * C::VFS];
    }
}

// Entropy projection of a batch's new state (Sec. 2.6): u (FP32 modal, in us
// as [field][mode][EPW]) -> u~ = u(Vh v_h) at the hybrid nodes, written to
// ut_out as float4 (h, u, v, H).  Mi: the element's packed (M_h^k)^{-1}
// (unused with the weight-adjusted inverse, which reads w J through wqv);
// ts, ss: scratch; bqv, wqv: b and w J at this lane's volume nodes q = b +
// LPE j; blv: b at its hybrid rows.  With the tensor-core contractions (C::TC)
// the state is in the warp's A operand instead of us, and ws is the warp's
// region.  Returns false if a bounded wait expired.
template <int N>
__device__ __forceinline__ bool stage2_project(const StageParams<float>& p, float* __restrict__ ut_out,
                                               const float* __restrict__ ops, const float* Mi, const float* us,
                                               float* ts, float* ss, int ge, int lane,
                                               const float (&bqv)[C2<N>::QPL], const float (&wqv)[C2<N>::QPL],
                                               const float (&blv)[C2<N>::RPL], float* ws = nullptr) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL, QPL = C::QPL, MPL = C::MPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const float g = p.g;
    const float ig = 1.f / g;
    const bool valid = ge < p.K;
    int bad = 0;
    float v0[RPL], v1[RPL], v2[RPL];
    if constexpr (C::TC) {
        tc_project<N>(p, ops, Mi, ws, ge, lane, bqv, wqv, v0, v1, v2, bad);
    } else {
        // ---- entropy projection of the new state: u_q = Vq u, v(u_q) w J -------
        {
            float q0[QPL], q1[QPL], q2[QPL];
#pragma unroll
            for (int j = 0; j < QPL; ++j) q0[j] = q1[j] = q2[j] = 0.f;
            for (int n = 0; n < D::Np; ++n) {
                const float u0 = us[(0 * D::Np + n) * EPW + e];
                const float u1 = us[(1 * D::Np + n) * EPW + e];
                const float u2 = us[(2 * D::Np + n) * EPW + e];
                const float* v = ops + C::o_Vq + (n * LPE + b) * C::QPLp;
#pragma unroll
                for (int j = 0; j < QPL; ++j) {
                    q0[j] = fmaf(v[j], u0, q0[j]);
                    q1[j] = fmaf(v[j], u1, q1[j]);
                    q2[j] = fmaf(v[j], u2, q2[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < QPL; ++j) {
                const int q = b + LPE * j;
                if (q < D::Nq) {
                    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
                    if (valid) {
                        const float h = q0[j];
                        if (!(h > 0.f)) bad |= STATUS_NONPOSITIVE;
                        const float ih = 1.f / h;
                        const float uu = q1[j] * ih, vv = q2[j] * ih;
                        const float wj = wqv[j];
                        t0 = wj * (g * (h + bqv[j]) - 0.5f * (uu * uu + vv * vv));
                        t1 = wj * uu;
                        t2 = wj * vv;
                    }
                    ts[(0 * D::Nq + q) * EPW + e] = t0;
                    ts[(1 * D::Nq + q) * EPW + e] = t1;
                    ts[(2 * D::Nq + q) * EPW + e] = t2;
                }
            }
        }
        __syncwarp();
        if constexpr (C::WADG) {
            // weight-adjusted: z = (w/J) o (A (w J v)) at the volume nodes q = b + LPE*j
            float c0[QPL], c1[QPL], c2[QPL];
#pragma unroll
            for (int j = 0; j < QPL; ++j) c0[j] = c1[j] = c2[j] = 0.f;
            for (int q2 = 0; q2 < D::Nq; ++q2) {
                const float t0 = ts[(0 * D::Nq + q2) * EPW + e];
                const float t1 = ts[(1 * D::Nq + q2) * EPW + e];
                const float t2 = ts[(2 * D::Nq + q2) * EPW + e];
                const float* v = ops + C::o_A + (q2 * LPE + b) * C::QPLp;
#pragma unroll
                for (int j = 0; j < QPL; ++j) {
                    c0[j] = fmaf(v[j], t0, c0[j]);
                    c1[j] = fmaf(v[j], t1, c1[j]);
                    c2[j] = fmaf(v[j], t2, c2[j]);
                }
            }
            __syncwarp();  // every lane has read w J v
#pragma unroll
            for (int j = 0; j < QPL; ++j) {
                const int q = b + LPE * j;
                if (q < D::Nq) {
                    const float w = ops[C::o_wq + q];
                    const float sc = valid ? w * w / wqv[j] : 0.f;
                    ts[(0 * D::Nq + q) * EPW + e] = c0[j] * sc;
                    ts[(1 * D::Nq + q) * EPW + e] = c1[j] * sc;
                    ts[(2 * D::Nq + q) * EPW + e] = c2[j] * sc;
                }
            }
            __syncwarp();
            // v~ = B z at the hybrid nodes l = b + LPE*j
#pragma unroll
            for (int j = 0; j < RPL; ++j) v0[j] = v1[j] = v2[j] = 0.f;
            for (int q = 0; q < D::Nq; ++q) {
                const float z0 = ts[(0 * D::Nq + q) * EPW + e];
                const float z1 = ts[(1 * D::Nq + q) * EPW + e];
                const float z2 = ts[(2 * D::Nq + q) * EPW + e];
                const float* v = ops + C::o_B + (q * LPE + b) * C::RPLp;
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    v0[j] = fmaf(v[j], z0, v0[j]);
                    v1[j] = fmaf(v[j], z1, v1[j]);
                    v2[j] = fmaf(v[j], z2, v2[j]);
                }
            }
        } else {
            // y = Vq^T (w J v), modes n = b + LPE*j
            {
                float y0[MPL], y1[MPL], y2[MPL];
#pragma unroll
                for (int j = 0; j < MPL; ++j) y0[j] = y1[j] = y2[j] = 0.f;
                for (int q = 0; q < D::Nq; ++q) {
                    const float t0 = ts[(0 * D::Nq + q) * EPW + e];
                    const float t1 = ts[(1 * D::Nq + q) * EPW + e];
                    const float t2 = ts[(2 * D::Nq + q) * EPW + e];
                    const float* v = ops + C::o_VqT + (q * LPE + b) * C::MPLp;
#pragma unroll
                    for (int j = 0; j < MPL; ++j) {
                        y0[j] = fmaf(v[j], t0, y0[j]);
                        y1[j] = fmaf(v[j], t1, y1[j]);
                        y2[j] = fmaf(v[j], t2, y2[j]);
                    }
                }
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int n = b + LPE * j;
                    if (n < D::Np) {
                        ss[(0 * D::Np + n) * EPW + e] = y0[j];
                        ss[(1 * D::Np + n) * EPW + e] = y1[j];
                        ss[(2 * D::Np + n) * EPW + e] = y2[j];
                    }
                }
            }
            __syncwarp();
            // v_h = (M_h^k)^{-1} y, in place (modes n = b + LPE*j)
            {
                float r0[MPL], r1[MPL], r2[MPL];
                minv_rows<D::Np, MPL, LPE, EPW>(Mi, ss + e, b, r0, r1, r2);
                __syncwarp();
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int n = b + LPE * j;
                    if (n < D::Np) {
                        ss[(0 * D::Np + n) * EPW + e] = r0[j];
                        ss[(1 * D::Np + n) * EPW + e] = r1[j];
                        ss[(2 * D::Np + n) * EPW + e] = r2[j];
                    }
                }
            }
            __syncwarp();
            // v~ = Vh v_h at the hybrid nodes l = b + LPE*j
#pragma unroll
            for (int j = 0; j < RPL; ++j) v0[j] = v1[j] = v2[j] = 0.f;
            for (int n = 0; n < D::Np; ++n) {
                const float w0 = ss[(0 * D::Np + n) * EPW + e];
                const float w1 = ss[(1 * D::Np + n) * EPW + e];
                const float w2 = ss[(2 * D::Np + n) * EPW + e];
                const float* v = ops + C::o_Vh + (n * LPE + b) * C::RPLp;
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    v0[j] = fmaf(v[j], w0, v0[j]);
                    v1[j] = fmaf(v[j], w1, v1[j]);
                    v2[j] = fmaf(v[j], w2, v2[j]);
                }
            }
        }
    }
    // u~ = u(v~), stored as (h, u, v, H - H_0): the free surface relative to
    // the element's first hybrid node, which only the element's own next stage
    // reads (the pressure terms of stage2_batch; neighbours read h, u, v)
    {
        const float H_j0 = (v0[0] + 0.5f * (v1[0] * v1[0] + v2[0] * v2[0])) * ig;  // row l = b
        const float H0 = __shfl_sync(0xffffffffu, H_j0, lane & ~(LPE - 1));      // row 0 of the element
        if (valid) {
#pragma unroll
            for (int j = 0; j < RPL; ++j) {
                const int l = b + LPE * j;
                if (l < D::Nh) {
                    const float H = (v0[j] + 0.5f * (v1[j] * v1[j] + v2[j] * v2[j])) * ig;
                    const float h = H - blv[j];
                    if (!(h > 0.f)) bad |= STATUS_NONPOSITIVE;
                    if (!isfinite(H) || !isfinite(v1[j]) || !isfinite(v2[j])) bad |= STATUS_NONFINITE;
                    *reinterpret_cast<float4*>(ut_out + ((size_t)ge * D::Nh + l) * 4) =
                        make_float4(h, v1[j], v2[j], H - H0);
                }
            }
        }
    }
    if (bad) atomicOr(p.status, bad);
    return true;
}

// Host-state calls: the batch's new FP64 state, just written to p.u at each
// lane's modes, copied to the caller's (host-resident) u_out in contiguous
// runs (j = lane + 32 k in [field][element][mode] order): writes over the host
// link in whole 256-byte runs rather than 64-byte pieces.
template <int N>
__device__ __forceinline__ void copy_state_out(const StageParams<float>& p, double* u_out, int e0, int lane) {
    typedef Dims<N> D;
    constexpr int EPW = C2<N>::EPW, NRK = 3 * EPW * D::Np;
    __syncwarp();  // the warp's writes of p.u are visible to its lanes
    for (int j = lane; j < NRK; j += 32) {
        const int c = j / (EPW * D::Np), o = j - c * (EPW * D::Np);
        if (e0 + o / D::Np < p.K) {
            const size_t gi = ((size_t)c * p.K + e0) * D::Np + o;
            u_out[gi] = p.u[gi];
        }
    }
}

// The manufactured-solution forcing of Sec. 4.1 (sine solution) at volume
// node q of element ge, J-weighted: w J f.
template <int N>
__device__ __forceinline__ void mms_forcing_at(const StageParams<float>& p, int ge, int q, float& f0, float& f1,
                                               float& f2) {
    typedef Dims<N> D;
    const float g = p.g;
    const float x = p.xq[(size_t)ge * D::Nq + q], y = p.yq[(size_t)ge * D::Nq + q];
    const float wj = p.wJq[(size_t)ge * D::Nq + q];
    float sth, cth, sx, cx, sy, cy;
    sincospif(x + y - (float)p.t, &sth, &cth);
    sincospif(x, &sx, &cx);
    sincospif(y, &sy, &cy);
    const float pi = 3.14159265358979323846f;
    const float h = 2.f + p.mms_amp * sth;
    const float cc = p.mms_amp * pi * cth;
    const float bx = -p.mms_bamp * pi * sx * cy, by = -p.mms_bamp * pi * cx * sy;
    const float u0 = p.mms_u0, v0 = p.mms_v0;
    f0 = wj * (-cc + u0 * cc + v0 * cc);
    f1 = wj * (-u0 * cc + (u0 * u0 + g * h) * cc + u0 * v0 * cc + g * h * bx);
    f2 = wj * (-v0 * cc + u0 * v0 * cc + (v0 * v0 + g * h) * cc + g * h * by);
}

// The rest of a batch after the volume and interface phase, with the dense
// contractions on the tensor cores: the lift s = Vh^T r - Vq^T (W J f) (MMA),
// du/dt = -(M_h^k)^{-1} s (FP32 pipes, modes n = b + LPE j of each lane),
// then du/dt out (MODE 0) or the LSRK45 stage in FP64 on the same lanes and
// the entropy projection of the new state (MODE 1).  a0..a2: the rows
// l = b + LPE i of the volume and interface terms.
template <int N, int MODE>
__device__ __forceinline__ void tc_batch_tail(const StageParams<float>& p, float* __restrict__ ut_out, double rkA,
                                              double rkB, const float* __restrict__ ops, float* ws, int e0, int lane,
                                              const float (&a0)[C2<N>::RPL], const float (&a1)[C2<N>::RPL],
                                              const float (&a2)[C2<N>::RPL]) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL, QPL = C::QPL, MPL = C::MPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const int K = p.K;
    const int ge = e0 + e;
    const bool valid = ge < K;
    float* tA = ws + C::t_A;
    float* tin = ws + C::t_in;
    const float* tb = ops + C::o_tc;
    const float* Mi = ws + C::w_mi + e * C::MIS;
    int of[3];
#pragma unroll
    for (int f = 0; f < 3; ++f) of[f] = tc_off(3 * e + f, b);
    // the volume and face rows as the A operand of the lift (zero past Nh)
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        if (b + LPE * i < C::KL) {
            const bool in = b + LPE * i < D::Nh;
            tc_put_at(tA, C::KL, of[0] + 128 * i, in ? a0[i] : 0.f);
            tc_put_at(tA, C::KL, of[1] + 128 * i, in ? a1[i] : 0.f);
            tc_put_at(tA, C::KL, of[2] + 128 * i, in ? a2[i] : 0.f);
        }
    }
    float d[16] = {};
    if (!p.forcing) {
        tc_round<N, C::KL>(tA, tb + C::tb_lift, tb + C::tb_lift + C::NpR * C::KL, false, p.status, lane, d);
    } else {
        tc_round<N, C::KL, false>(tA, tb + C::tb_lift, tb + C::tb_lift + C::NpR * C::KL, false, p.status, lane, d);
        // the lift's operand is consumed: -W J f over the volume nodes, accumulated
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = b + LPE * j;
            if (q < C::KQ) {
                float f0 = 0.f, f1 = 0.f, f2 = 0.f;
                if (valid && q < D::Nq) mms_forcing_at<N>(p, ge, q, f0, f1, f2);
                tc_put_at(tA, C::KQ, of[0] + 128 * j, -f0);
                tc_put_at(tA, C::KQ, of[1] + 128 * j, -f1);
                tc_put_at(tA, C::KQ, of[2] + 128 * j, -f2);
            }
        }
        tc_round<N, C::KQ>(tA, tb + C::tb_vqt, tb + C::tb_vqt + C::NpR * C::KQ, true, p.status, lane, d);
    }
    tc_store_rows<EPW>(tin, C::TES, C::TFS, lane, d);
    __syncwarp();
    float r0[MPL], r1[MPL], r2[MPL];
    minv_rows<D::Np, MPL, LPE, EPW, C::TFS, 1>(Mi, tin + e * C::TES, b, r0, r1, r2);
    const float* rr[3] = {r0, r1, r2};
    if constexpr (MODE == 0) {
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int n = b + LPE * j;
                if (valid && n < D::Np) p.rhs_out[((size_t)f * K + ge) * D::Np + n] = (double)(-rr[f][j]);
            }
        return;
    }
    // b and w J at this lane's nodes for the projection
    float bqv[QPL], wqv[QPL], blv[RPL];
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = b + LPE * j;
        bqv[j] = wqv[j] = 0.f;
        if (valid && q < D::Nq) {
            bqv[j] = __ldg(p.bh + (size_t)ge * D::Nh + q);
            wqv[j] = __ldg(p.wJq + (size_t)ge * D::Nq + q);
        }
    }
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int l = b + LPE * j;
        blv[j] = (valid && l < D::Nh) ? __ldg(p.bh + (size_t)ge * D::Nh + l) : 0.f;
    }
    // LSRK45 stage in FP64 at the lane's modes: res = A res + dt du/dt,
    // u += B res; the new FP32 state as the A operand of u_q = Vq u (zero past Np)
    const float dtf = (float)p.dt;
    double* const u_out = p.u_out;  // host-state calls: the last stage also writes the state there
#pragma unroll
    for (int f = 0; f < 3; ++f)
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            const int n = b + LPE * j;
            double un = 1.0;
            if (valid && n < D::Np) {
                const size_t gi = ((size_t)f * K + ge) * D::Np + n;
                const double r = rkA != 0.0 ? p.res[gi] : 0.0;  // the first LSRK45 stage (A = 0) does not read it
                const double rs = fma(rkA, r, f2d_bits(dtf * (-rr[f][j])));
                un = fma(rkB, rs, p.u[gi]);
                p.res[gi] = rs;
                p.u[gi] = un;
            }
            tc_put_at(tA, C::KM, of[f] + 128 * j, n < D::Np ? d2f_bits(un) : 0.f);
        }
    if (u_out) copy_state_out<N>(p, u_out, e0, lane);
    stage2_project<N>(p, ut_out, ops, Mi, nullptr, nullptr, nullptr, ge, lane, bqv, wqv, blv, ws);
}

// Volume flux differencing with unique pairs (C2::UP): the row data of this
// lane's slots (volume slots loaded first, face slots after the pair loops,
// which do not read them) and the accumulators a0..a2 of every slot, before
// the row part u_l sum(T) is added.  The arithmetic of a pair is that of the
// ordered loop from row l's side; row m receives -T for h and, for the
// momenta, -(u_l T + Qx 2 g h_m (H_l - H_0)) (the partner's column is l), as
// the ordered loop would have formed them from row m's side.
template <int N>
__device__ __forceinline__ void stage2_unique_pairs(const float* __restrict__ ops, const float4* utE,
                                                    const float4* geE, int b, float g, float* rh, float* ru,
                                                    float* rv, float* rrx, float* rsx, float* rry, float* rsy,
                                                    float* a0, float* a1, float* a2) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, RPL = C::RPL, VS = C::VS;
    static_assert(VS == 2, "two volume row slots a lane (one float4 of entries per partner row)");
    float rH[VS];
#pragma unroll
    for (int i = 0; i < RPL; ++i) a0[i] = a1[i] = a2[i] = 0.f;
#pragma unroll
    for (int i = 0; i < VS; ++i) {
        const float4 U = utE[b + LPE * i], G = geE[b + LPE * i];
        rh[i] = U.x;
        ru[i] = U.y;
        rv[i] = U.z;
        rH[i] = U.w;
        rrx[i] = G.x;
        rsx[i] = G.y;
        rry[i] = G.z;
        rsy[i] = G.w;
    }
    const float g2 = 2.f * g;
    // own row slot I against the partner row whose records are U, G; c0..c2
    // collect the partner row's share (subtracted by the receiver)
#define ESDG_UPAIR(I, QR, QS, FIRST)                                           \
{                                                                          \
    const float Qx = (QR) * (rrx[I] + G.x) + (QS) * (rsx[I] + G.y);        \
    const float Qy = (QR) * (rry[I] + G.z) + (QS) * (rsy[I] + G.w);        \
    const float HU = fmaf(rh[I], ru[I], hum), HV = fmaf(rh[I], rv[I], hvm);\
    const float T = fmaf(Qx, HU, Qy * HV);                                 \
    const float Pl = rh[I] * gH2, Pm = hm2 * rH[I];                        \
    a0[I] += T;                                                            \
    a1[I] = fmaf(U.y, T, fmaf(Qx, Pl, a1[I]));                             \
    a2[I] = fmaf(U.z, T, fmaf(Qy, Pl, a2[I]));                             \
    if (FIRST) {                                                           \
        c0 = T;                                                            \
        c1 = fmaf(ru[I], T, Qx * Pm);                                      \
        c2 = fmaf(rv[I], T, Qy * Pm);                                      \
    } else {                                                               \
        c0 += T;                                                           \
        c1 = fmaf(ru[I], T, fmaf(Qx, Pm, c1));                             \
        c2 = fmaf(rv[I], T, fmaf(Qy, Pm, c2));                             \
    }                                                                      \
}
    // offset 0, volume-volume: rows b and b + LPE of this lane
    {
        const float2 q = *reinterpret_cast<const float2*>(ops + C::o_U0 + 2 * b);
        const float4 U = make_float4(rh[1], ru[1], rv[1], rH[1]);
        const float4 G = make_float4(rrx[1], rsx[1], rry[1], rsy[1]);
        const float hum = U.x * U.y, hvm = U.x * U.z, gH2 = g2 * U.w, hm2 = g2 * U.x;
        float c0, c1, c2;
        ESDG_UPAIR(0, q.x, q.y, true)
        a0[1] -= c0;
        a1[1] -= c1;
        a2[1] -= c2;
    }
    // partner slot J at offset s: the partner row m = (b + s) mod LPE + LPE J
    // (clamped into the element's rows; its entries are zero past Nh), and
    // the share of this lane's slot J from lane (b - s) mod LPE
#define ESDG_USTEP(TABLE, J)                                                   \
{                                                                          \
    const int m = min(((b + s) & (LPE - 1)) + LPE * (J), D::Nh - 1);       \
    const float4 U = utE[m], G = geE[m];                                   \
    const float4 q = *reinterpret_cast<const float4*>(TABLE + 4 * b);      \
    const float hum = U.x * U.y, hvm = U.x * U.z, gH2 = g2 * U.w, hm2 = g2 * U.x; \
    float c0, c1, c2;                                                      \
    ESDG_UPAIR(0, q.x, q.y, true)                                          \
    ESDG_UPAIR(1, q.z, q.w, false)                                         \
    const int src = (b - s) & (LPE - 1);                                   \
    a0[J] -= __shfl_sync(0xffffffffu, c0, src, LPE);                       \
    a1[J] -= __shfl_sync(0xffffffffu, c1, src, LPE);                       \
    a2[J] -= __shfl_sync(0xffffffffu, c2, src, LPE);                       \
}
#pragma unroll 2
    for (int s = 1; s <= LPE / 2; ++s) {
        const float* t = ops + C::o_Uvv + (s - 1) * VS * LPE * 4;
#pragma unroll
        for (int j = 0; j < VS; ++j) ESDG_USTEP(t + j * LPE * 4, j)
    }
#pragma unroll 1
    for (int s = 0; s < LPE; ++s) {
        const float* t = ops + C::o_Uvf + s * C::FS * LPE * 4;
#pragma unroll
        for (int j = VS; j < RPL; ++j) ESDG_USTEP(t + (j - VS) * LPE * 4, j)
    }
#undef ESDG_USTEP
#undef ESDG_UPAIR
#pragma unroll
    for (int i = VS; i < RPL; ++i) {
        const int l = b + LPE * i;
        float4 U = make_float4(0.f, 0.f, 0.f, 0.f), G = U;
        if (l < D::Nh) {
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
    }
}

// One batch of EPW elements of one problem, starting at element e0 (all 32
// lanes of the warp).  ops: the operator region of degree N in shared memory;
// ws: this warp's region.  Returns false if the bounded wait on the bulk
// copies expired (the status word then carries STATUS_TIMEOUT).
template <int N, int MODE>
__device__ __forceinline__ bool stage2_batch(const StageParams<float>& p, const float* __restrict__ ut_in,
                                             float* __restrict__ ut_out, double rkA, double rkB,
                                             const float* __restrict__ ops, float* ws, uint64_t* bar,
                                             uint32_t& parity, int e0, int lane) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL, QPL = C::QPL, MPL = C::MPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const float g = p.g;
    const int K = p.K;
    const int ge = e0 + e;
    const bool valid = ge < K;
    // ---- stage element data: TMA bulk copies (one per element and array) ----
    if (lane == 0) mbar_arrive_expect_tx(bar, C::TX_BYTES);
    __syncwarp();
    if (lane < (C::WADG ? 2 : 3) * EPW) {
        const int which = lane / EPW, ee = lane - which * EPW;
        if (which == 0)
            tma_bulk_g2s(ws + C::w_ut + ee * C::UTS, ut_in + (size_t)(e0 + ee) * D::Nh * 4, D::Nh * 16, bar);
        else if (which == 1)
            tma_bulk_g2s(ws + C::w_geo + ee * C::UTS, p.geo + (size_t)(e0 + ee) * D::Nh * 4, D::Nh * 16, bar);
        else
            tma_bulk_g2s(ws + C::w_mi + ee * C::MIS, p.minv + (size_t)(e0 + ee) * C::NpP4, C::NpP4 * 4, bar);
    }
    // neighbour traces of this batch (a gather: plain loads while the bulk copies fly)
    float4 tv[C::TRL];
    gather_traces<N>(p, ut_in, e0, lane, tv);
#pragma unroll
    for (int t = 0; t < C::TRL; ++t) {
        const int k = lane + 32 * t;
        if (k < EPW * D::Nfq) *reinterpret_cast<float4*>(ws + C::w_tr + k * 4) = tv[t];
    }
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, parity, p.status))) return false;
    parity ^= 1;
    __syncwarp();

    // ---- volume flux differencing, rows l = b + LPE*i ------------------------
    const float4* utE = reinterpret_cast<const float4*>(ws + C::w_ut + e * C::UTS);
    const float4* geE = reinterpret_cast<const float4*>(ws + C::w_geo + e * C::UTS);
    // Pressure and bathymetry enter as g h_l H_m (volume) and g h_l (h+ + b_l)
    // (interface).  Each row's operator satisfies sum_m Qskew[l,m] + B[l] = 0
    // (Q_h 1 = 0, the identity behind the lake-at-rest property of Theorem
    // 2.2), so a constant subtracted from every free surface H in both terms
    // leaves the exact right-hand side unchanged.  The records carry H - H_0,
    // H_0 the element's free surface at its first hybrid node (written by
    // stage2_project): the FP32 sums then no longer cancel large equal terms,
    // and the momentum error of the FP32 path falls about threefold.
    float rh[RPL], ru[RPL], rv[RPL], rrx[RPL], rsx[RPL], rry[RPL], rsy[RPL];
    float a0[RPL], a1[RPL], a2[RPL];
    if constexpr (C::UP) {
        stage2_unique_pairs<N>(ops, utE, geE, b, g, rh, ru, rv, rrx, rsx, rry, rsy, a0, a1, a2);
    } else {
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int l = b + LPE * i;
        float4 U = make_float4(0.f, 0.f, 0.f, 0.f), G = U;
        if (l < D::Nh) {
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
    // (u_l + u_m) T summed over m is u_l (sum of T) + sum of u_m T: the row
    // part is added once after the loop
#define ESDG_PAIR(I, QR, QS)                                                   \
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
#pragma unroll (C::VUNROLL)
    for (int m = 0; m < D::Nq; ++m) {
        const float4 U = utE[m], G = geE[m];
        const float hum = U.x * U.y, hvm = U.x * U.z, gH2 = 2.f * g * U.w;
        const float4* q4 = reinterpret_cast<const float4*>(QsB + m * LPE * C::OPB);
#pragma unroll
        for (int i2 = 0; i2 < (RPL + 1) / 2; ++i2) {
            const float4 q = q4[i2];
            ESDG_PAIR(2 * i2, q.x, q.y)
            if (2 * i2 + 1 < RPL) ESDG_PAIR(2 * i2 + 1, q.z, q.w)
        }
    }
#pragma unroll (C::VUNROLL)
    for (int m = D::Nq; m < D::Nh; ++m) {
        const float4 U = utE[m], G = geE[m];
        const float hum = U.x * U.y, hvm = U.x * U.z, gH2 = 2.f * g * U.w;
        const float4* q4 = reinterpret_cast<const float4*>(QsB + m * LPE * C::OPB);
#pragma unroll
        for (int i2 = 0; i2 < (RPL + 1) / 2; ++i2) {
            if (LPE * (2 * i2) < D::Nq) {
                const float4 q = q4[i2];
                // face rows (l >= Nq) have no face columns; their entries are zero,
                // so the predicate only skips work
                if (b + LPE * (2 * i2) < D::Nq) ESDG_PAIR(2 * i2, q.x, q.y)
                if (2 * i2 + 1 < RPL && b + LPE * (2 * i2 + 1) < D::Nq) ESDG_PAIR(2 * i2 + 1, q.z, q.w)
            }
        }
    }
#undef ESDG_PAIR
    }
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        a1[i] = fmaf(ru[i], a0[i], a1[i]);
        a2[i] = fmaf(rv[i], a0[i], a2[i]);
    }
    // ---- interface flux on the face rows ------------------------------------
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        a0[i] *= 2.f;
        const int l = b + LPE * i;
        if (LPE * i + LPE - 1 >= D::Nq && l >= D::Nq && l < D::Nh) {
            const int f = l - D::Nq;
            const float4 U = utE[l];
            const float4 tp = *reinterpret_cast<const float4*>(ws + C::w_tr + (e * D::Nfq + f) * 4);
            const float h_l = U.x;
            const float nr = ops[C::o_nrs + 2 * f], ns = ops[C::o_nrs + 2 * f + 1];
            const float nxJ = 8.f * (rrx[i] * nr + rsx[i] * ns);
            const float nyJ = 8.f * (rry[i] * nr + rsy[i] * ns);
            float hP = tp.x, uP = tp.y, vP = tp.z;
            if (p.walls && (__ldg(p.nbr + (size_t)ge * 3 + f / D::Nfp) & 3) == 3) {
                // reflective wall (Sec. 2.9): h+ = h, u_n+ = -u_n, tangential kept
                const float sJw = sqrtf(nxJ * nxJ + nyJ * nyJ);
                const float wnx = nxJ / sJw, wny = nyJ / sJw;
                const float un = ru[i] * wnx + rv[i] * wny;
                hP = h_l;
                uP = ru[i] - 2.f * un * wnx;
                vP = rv[i] - 2.f * un * wny;
            }
            const float huP = hP * uP, hvP = hP * vP;
            const float w = ops[C::o_wf + f];
            const float hu_l = h_l * ru[i], hv_l = h_l * rv[i];
            const float huA = 0.5f * (hu_l + huP), hvA = 0.5f * (hv_l + hvP);
            const float uA = 0.5f * (ru[i] + uP), vA = 0.5f * (rv[i] + vP);
            const float pw = 0.5f * g * h_l * ((hP - h_l) + U.w);  // (h+ + b_l) - H_0
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
    }
    __syncwarp();  // every lane is done with the u~ / metric staging
    if constexpr (C::TC) {
        tc_batch_tail<N, MODE>(p, ut_out, rkA, rkB, ops, ws, e0, lane, a0, a1, a2);
    } else {
    float* rt = ws + C::s_rt;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
        const int l = b + LPE * i;
        if (l < D::Nh) {
            rt[(0 * D::Nh + l) * EPW + e] = a0[i];
            rt[(1 * D::Nh + l) * EPW + e] = a1[i];
            rt[(2 * D::Nh + l) * EPW + e] = a2[i];
        }
    }
    // The FP64 RK state: at this lane's element and modes n = b + LPE j (the
    // modes whose du/dt the inverse mass leaves in this lane's registers;
    // C::RK_LANES), or spread over all 32 lanes (j = lane + 32 k in
    // [field][element][mode] order, contiguous per field in global memory).
    // Loaded here, so that the latency overlaps the lift and the inverse mass,
    // where the registers allow it (C::EARLY_RK); otherwise just before the
    // update (1.2% faster at N = 4 with the stored inverse; 2% slower where
    // the early loads fit).
    constexpr int NRK = 3 * EPW * D::Np;
    constexpr int RKV = C::RK_LANES ? 3 * MPL : C::RKL;
    double uj[RKV], rj[RKV];
    auto load_rk = [&]() {
        if constexpr (C::RK_LANES) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int n = b + LPE * j;
                    uj[f * MPL + j] = 0.0;
                    rj[f * MPL + j] = 0.0;
                    if (valid && n < D::Np) {
                        const size_t gi = ((size_t)f * K + ge) * D::Np + n;
                        uj[f * MPL + j] = p.u[gi];
                        if (rkA != 0.0) rj[f * MPL + j] = p.res[gi];  // the first LSRK45 stage (A = 0) does not read it
                    }
                }
        } else {
#pragma unroll
            for (int k = 0; k < C::RKL; ++k) {
                const int j = lane + 32 * k;
                uj[k] = 0.0;
                rj[k] = 0.0;
                if (j < NRK) {
                    const int c = j / (EPW * D::Np), o = j - c * (EPW * D::Np);
                    if (e0 + o / D::Np < K) {
                        const size_t gi = ((size_t)c * K + e0) * D::Np + o;
                        uj[k] = p.u[gi];
                        if (rkA != 0.0) rj[k] = p.res[gi];
                    }
                }
            }
        }
    };
    if (MODE == 1 && C::EARLY_RK) load_rk();
    // forcing at the volume nodes, J-weighted (added as + Vq^T W J f)
    float* ts = ws + C::s_t;
    auto forcing_at = [&](int q, float& f0, float& f1, float& f2) {
        f0 = f1 = f2 = 0.f;
        if (valid && q < D::Nq) mms_forcing_at<N>(p, ge, q, f0, f1, f2);
    };
    if (p.forcing) {
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = b + LPE * j;
            if (q < D::Nq) {
                float f0, f1, f2;
                forcing_at(q, f0, f1, f2);
                ts[(0 * D::Nq + q) * EPW + e] = f0;
                ts[(1 * D::Nq + q) * EPW + e] = f1;
                ts[(2 * D::Nq + q) * EPW + e] = f2;
            }
        }
    }
    __syncwarp();
    float* ss = ws + C::s_s;
    float du[3][MPL];  // du/dt at this lane's modes n = b + LPE j
    float bqv[QPL], wqv[QPL], blv[RPL];
    const float* Mi = ws + C::w_mi + e * C::MIS;  // the stored inverse (unused when weight-adjusted)
    if constexpr (C::WADG) {
        // ---- weight-adjusted: du/dt = -Vq^T [(w/J) o (C rt - A (w J f))] -------
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = b + LPE * j;
            wqv[j] = (valid && q < D::Nq) ? __ldg(p.wJq + (size_t)ge * D::Nq + q) : 0.f;
        }
        float c0[QPL], c1[QPL], c2[QPL];
#pragma unroll
        for (int j = 0; j < QPL; ++j) c0[j] = c1[j] = c2[j] = 0.f;
        for (int l = 0; l < D::Nh; ++l) {
            const float r0 = rt[(0 * D::Nh + l) * EPW + e];
            const float r1 = rt[(1 * D::Nh + l) * EPW + e];
            const float r2 = rt[(2 * D::Nh + l) * EPW + e];
            const float* v = ops + C::o_C + (l * LPE + b) * C::QPLp;
#pragma unroll
            for (int j = 0; j < QPL; ++j) {
                c0[j] = fmaf(v[j], r0, c0[j]);
                c1[j] = fmaf(v[j], r1, c1[j]);
                c2[j] = fmaf(v[j], r2, c2[j]);
            }
        }
        if (p.forcing) {
            for (int q2 = 0; q2 < D::Nq; ++q2) {
                const float f0 = ts[(0 * D::Nq + q2) * EPW + e];
                const float f1 = ts[(1 * D::Nq + q2) * EPW + e];
                const float f2 = ts[(2 * D::Nq + q2) * EPW + e];
                const float* v = ops + C::o_A + (q2 * LPE + b) * C::QPLp;
#pragma unroll
                for (int j = 0; j < QPL; ++j) {
                    c0[j] = fmaf(-v[j], f0, c0[j]);
                    c1[j] = fmaf(-v[j], f1, c1[j]);
                    c2[j] = fmaf(-v[j], f2, c2[j]);
                }
            }
        }
        __syncwarp();  // every lane has read the forcing
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = b + LPE * j;
            if (q < D::Nq) {
                const float w = ops[C::o_wq + q];
                const float sc = valid ? w * w / wqv[j] : 0.f;
                ts[(0 * D::Nq + q) * EPW + e] = c0[j] * sc;
                ts[(1 * D::Nq + q) * EPW + e] = c1[j] * sc;
                ts[(2 * D::Nq + q) * EPW + e] = c2[j] * sc;
            }
        }
        __syncwarp();
        float r0[MPL], r1[MPL], r2[MPL];
#pragma unroll
        for (int j = 0; j < MPL; ++j) r0[j] = r1[j] = r2[j] = 0.f;
        for (int q = 0; q < D::Nq; ++q) {
            const float z0 = ts[(0 * D::Nq + q) * EPW + e];
            const float z1 = ts[(1 * D::Nq + q) * EPW + e];
            const float z2 = ts[(2 * D::Nq + q) * EPW + e];
            const float* v = ops + C::o_VqT + (q * LPE + b) * C::MPLp;
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                r0[j] = fmaf(v[j], z0, r0[j]);
                r1[j] = fmaf(v[j], z1, r1[j]);
                r2[j] = fmaf(v[j], z2, r2[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < MPL; ++j) {
            du[0][j] = -r0[j];
            du[1][j] = -r1[j];
            du[2][j] = -r2[j];
        }
    } else {
        // ---- lift: s = Vh^T rt - Vq^T W J f, modes n = b + LPE*j --------------
        {
            float s0[MPL], s1[MPL], s2[MPL];
#pragma unroll
            for (int j = 0; j < MPL; ++j) s0[j] = s1[j] = s2[j] = 0.f;
            for (int l = 0; l < D::Nh; ++l) {
                const float r0 = rt[(0 * D::Nh + l) * EPW + e];
                const float r1 = rt[(1 * D::Nh + l) * EPW + e];
                const float r2 = rt[(2 * D::Nh + l) * EPW + e];
                const float* v = ops + C::o_VhT + (l * LPE + b) * C::MPLp;
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    s0[j] = fmaf(v[j], r0, s0[j]);
                    s1[j] = fmaf(v[j], r1, s1[j]);
                    s2[j] = fmaf(v[j], r2, s2[j]);
                }
            }
            if (p.forcing) {
                for (int q = 0; q < D::Nq; ++q) {
                    const float f0 = ts[(0 * D::Nq + q) * EPW + e];
                    const float f1 = ts[(1 * D::Nq + q) * EPW + e];
                    const float f2 = ts[(2 * D::Nq + q) * EPW + e];
                    const float* v = ops + C::o_VqT + (q * LPE + b) * C::MPLp;
#pragma unroll
                    for (int j = 0; j < MPL; ++j) {
                        s0[j] = fmaf(-v[j], f0, s0[j]);
                        s1[j] = fmaf(-v[j], f1, s1[j]);
                        s2[j] = fmaf(-v[j], f2, s2[j]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int n = b + LPE * j;
                if (n < D::Np) {
                    ss[(0 * D::Np + n) * EPW + e] = s0[j];
                    ss[(1 * D::Np + n) * EPW + e] = s1[j];
                    ss[(2 * D::Np + n) * EPW + e] = s2[j];
                }
            }
        }
        __syncwarp();
        // ---- du/dt = -(M_h^k)^{-1} s at the lane's modes n = b + LPE*j, in registers
        {
            float r0[MPL], r1[MPL], r2[MPL];
            minv_rows<D::Np, MPL, LPE, EPW>(Mi, ss + e, b, r0, r1, r2);
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                du[0][j] = -r0[j];
                du[1][j] = -r1[j];
                du[2][j] = -r2[j];
            }
        }
    }
    __syncwarp();
    float* us = ws + C::s_u;
    // b and w J at this lane's nodes for the projection, loaded before the RK
    // update so their latency overlaps it
    if (MODE == 1) {
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = b + LPE * j;
            bqv[j] = 0.f;
            if (!C::WADG) wqv[j] = 0.f;
            if (valid && q < D::Nq) {
                bqv[j] = __ldg(p.bh + (size_t)ge * D::Nh + q);
                if (!C::WADG) wqv[j] = __ldg(p.wJq + (size_t)ge * D::Nq + q);
            }
        }
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int l = b + LPE * j;
            blv[j] = (valid && l < D::Nh) ? __ldg(p.bh + (size_t)ge * D::Nh + l) : 0.f;
        }
    }
    if constexpr (!C::RK_LANES) {
        // du/dt into ss as [field][element][mode] for the spread-out update
        __syncwarp();  // every lane has read s (the inverse mass's input aliases ss)
#pragma unroll
        for (int f = 0; f < 3; ++f)
#pragma unroll
            for (int j = 0; j < MPL; ++j) {
                const int n = b + LPE * j;
                if (n < D::Np) ss[(f * EPW + e) * D::Np + n] = du[f][j];
            }
        __syncwarp();
    }
    if (MODE == 0) {
        if constexpr (C::RK_LANES) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int n = b + LPE * j;
                    if (valid && n < D::Np) p.rhs_out[((size_t)f * K + ge) * D::Np + n] = (double)du[f][j];
                }
        } else {
            for (int j = lane; j < NRK; j += 32) {
                const int c = j / (EPW * D::Np), o = j - c * (EPW * D::Np);
                if (e0 + o / D::Np < K) p.rhs_out[((size_t)c * K + e0) * D::Np + o] = (double)ss[j];
            }
        }
    } else {
        // ---- LSRK45 stage in FP64: res = A res + dt rhs, u += B res
        if (!C::EARLY_RK) load_rk();
        const float dtf = (float)p.dt;
        double* const u_out = p.u_out;  // host-state calls: the last stage also writes the state there
        if constexpr (C::RK_LANES) {
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int j = 0; j < MPL; ++j) {
                    const int n = b + LPE * j;
                    if (n < D::Np) {
                        double un = 1.0;
                        if (valid) {
                            const size_t gi = ((size_t)f * K + ge) * D::Np + n;
                            const double rs = fma(rkA, rj[f * MPL + j], f2d_bits(dtf * du[f][j]));
                            un = fma(rkB, rs, uj[f * MPL + j]);
                            p.res[gi] = rs;
                            p.u[gi] = un;
                        }
                        us[(f * D::Np + n) * EPW + e] = d2f_bits(un);
                    }
                }
            if (u_out) copy_state_out<N>(p, u_out, e0, lane);
        } else {
#pragma unroll
            for (int k = 0; k < C::RKL; ++k) {
                const int j = lane + 32 * k;
                if (j < NRK) {
                    const int c = j / (EPW * D::Np), o = j - c * (EPW * D::Np);
                    const int ee = o / D::Np, n = o - ee * D::Np;
                    double un = 1.0;
                    if (e0 + ee < K) {
                        const size_t gi = ((size_t)c * K + e0) * D::Np + o;
                        const double rs = fma(rkA, rj[k], f2d_bits(dtf * ss[j]));
                        un = fma(rkB, rs, uj[k]);
                        p.res[gi] = rs;
                        p.u[gi] = un;
                        if (u_out) u_out[gi] = un;
                    }
                    us[(c * D::Np + n) * EPW + ee] = d2f_bits(un);
                }
            }
        }
    }
    __syncwarp();
    if constexpr (MODE == 1) {
        if (!stage2_project<N>(p, ut_out, ops, Mi, us, ts, ss, ge, lane, bqv, wqv, blv, ws)) return false;
    }
    }
    // generic-proxy writes to the staging area must be ordered before the
    // next batch's bulk copies overwrite it
    fence_proxy_async_smem();
    __syncwarp();
    if constexpr (C::TC) return !tc_failed<N>();
    return true;
}

// Projection-only batch: u~ of the EPW elements starting at e0 from the FP64
// modal state p.u_in, into ut_out (the first u~ of a run of stages).
template <int N>
__device__ __forceinline__ bool project2_batch(const StageParams<float>& p, float* __restrict__ ut_out,
                                               const float* __restrict__ ops, float* ws, uint64_t* bar,
                                               uint32_t& parity, int e0, int lane) {
    typedef Dims<N> D;
    typedef C2<N> C;
    constexpr int LPE = C::LPE, EPW = C::EPW, RPL = C::RPL, QPL = C::QPL;
    const int e = lane / LPE, b = lane - (lane / LPE) * LPE;
    const int K = p.K;
    const int ge = e0 + e;
    const bool valid = ge < K;
    if constexpr (!C::WADG) {  // the stored inverse: one bulk copy per element
        if (lane == 0) mbar_arrive_expect_tx(bar, EPW * C::NpP4 * 4);
        __syncwarp();
        if (lane < EPW)
            tma_bulk_g2s(ws + C::w_mi + lane * C::MIS, p.minv + (size_t)(e0 + lane) * C::NpP4, C::NpP4 * 4, bar);
    }
    float bqv[QPL], wqv[QPL], blv[RPL];
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = b + LPE * j;
        bqv[j] = 0.f;
        wqv[j] = 0.f;
        if (valid && q < D::Nq) {
            bqv[j] = __ldg(p.bh + (size_t)ge * D::Nh + q);
            wqv[j] = __ldg(p.wJq + (size_t)ge * D::Nq + q);
        }
    }
#pragma unroll
    for (int j = 0; j < RPL; ++j) {
        const int l = b + LPE * j;
        blv[j] = (valid && l < D::Nh) ? __ldg(p.bh + (size_t)ge * D::Nh + l) : 0.f;
    }
    float* us = ws + C::s_u;
    constexpr int NRK = 3 * EPW * D::Np;
    for (int j = lane; j < NRK; j += 32) {
        const int c = j / (EPW * D::Np), o = j - c * (EPW * D::Np);
        const int ee = o / D::Np, n = o - ee * D::Np;
        const size_t gi = ((size_t)c * K + e0) * D::Np + o;
        const double un = e0 + ee < K ? p.u_in[gi] : 1.0;
        if constexpr (C::TC)
            tc_put(ws + C::t_A, C::KM, 3 * ee + c, n, d2f_bits(un));
        else
            us[(c * D::Np + n) * EPW + ee] = d2f_bits(un);
        if (p.copy_in && e0 + ee < K) {
            p.u[gi] = un;
            p.res[gi] = 0.0;
        }
    }
    if constexpr (C::TC) {
        if (lane < 3 * EPW)
            for (int n = D::Np; n < C::KM; ++n) tc_put(ws + C::t_A, C::KM, lane, n, 0.f);
    }
    if constexpr (!C::WADG) {
        if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, parity, p.status))) return false;
        parity ^= 1;
    }
    __syncwarp();
    if (!stage2_project<N>(p, ut_out, ops, ws + C::w_mi + e * C::MIS, us, ws + C::s_t, ws + C::s_s, ge, lane, bqv,
                           wqv, blv, ws))
        return false;
    fence_proxy_async_smem();
    __syncwarp();
    if constexpr (C::TC) return !tc_failed<N>();
    return true;
}

// MODE 0: du/dt into rhs_out; MODE 1: LSRK45 stage and projection of the new
// state; MODE 2: projection of p.u_in only.
template <int N, int MODE>
__global__ void __launch_bounds__(C2<N>::WARPS * 32, 1) k_stage2(StageParams<float> p, const float* __restrict__ ops2, int Kpad) {
    typedef C2<N> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* ops = reinterpret_cast<float*>(smem_raw);
    const int nwarps = blockDim.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ops + C::o_end + nwarps * C::w_end);
    for (int i = threadIdx.x; i < C::o_end / 4; i += blockDim.x)
        reinterpret_cast<float4*>(ops)[i] = reinterpret_cast<const float4*>(ops2)[i];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) mbar_init(&bars[warp], 1);
    // tensor cores: one MMA-completion barrier per warp, and 512 TMEM columns
    // for the block (one block per SM), 16 for each warp
    if constexpr (C::TC) {
        if (lane == 0) {
            mbar_init(reinterpret_cast<uint64_t*>(smem_raw + C::tc_bar) + warp, 1);
            reinterpret_cast<uint32_t*>(smem_raw + C::tc_par)[warp] = 0u;
        }
        if (warp == 0) tc_alloc(smem_u32(smem_raw + C::tc_slot), 512);
    }
    fence_mbar_init();
    if constexpr (C::TC) tc_fence_before();
    __syncthreads();
    if constexpr (C::TC) tc_fence_after();
    uint64_t* bar = &bars[warp];
    float* ws = ops + C::o_end + warp * C::w_end;
    uint32_t parity = 0;
    // Warps that share a scheduler (warp, warp + 4, ...) start a fraction of a
    // batch apart, so their memory-latency phases do not coincide (identical
    // per-batch work otherwise keeps them in lockstep).
    __nanosleep((unsigned)(warp >> 2) * 1300u);
    const int nbatch = Kpad / C::EPW;
    for (int batch = blockIdx.x * nwarps + warp; batch < nbatch; batch += gridDim.x * nwarps) {
        bool ok;
        if constexpr (MODE == 2)
            ok = project2_batch<N>(p, p.ut_out, ops, ws, bar, parity, batch * C::EPW, lane);
        else
            ok = stage2_batch<N, MODE>(p, p.ut_in, p.ut_out, p.rkA, p.rkB, ops, ws, bar, parity, batch * C::EPW,
                                       lane);
        if (!ok) break;  // a bounded wait expired (status set)
    }
    if constexpr (C::TC) {
        // every warp's MMAs have completed (each waited for its own; after an
        // expired wait, once more with a bound); free the tensor memory
        if (tc_failed<N>()) {
            const long long t1 = clock64();
            while (!mbar_try_wait(tc_bar_of_warp<N>(), *tc_state_of_warp<N>() & 1u) && clock64() - t1 < (1LL << 31)) {
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 0) tc_dealloc(*reinterpret_cast<const uint32_t*>(smem_raw + C::tc_slot), 512);
    }
}

}  // namespace esdg
