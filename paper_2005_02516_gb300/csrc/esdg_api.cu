// C ABI of the ESDG shallow-water library (see include/esdg.h).
// Host set-up builds the FP64 operators and geometry once (host_build.cpp);
// all per-stage work runs in the kernels of esdg_kernels.cuh.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "esdg.h"
#include "esdg_launch.hpp"
#include "esdg_sbp2.cuh"
#include "host_build.hpp"

namespace esdg {

// Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage coefficients
// (the integrator of Sec. 4).
static const double RK_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                               -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double RK_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                               1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                               2277821191437.0 / 14882151754819.0};
static const double RK_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                               2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

__global__ void k_entropy_finalize(int nparts, const double* __restrict__ partial, double* __restrict__ out) {
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int i = 0; i < nparts; ++i) s += partial[i * 3 + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

}  // namespace esdg

using namespace esdg;

// Device memory map (offsets into one buffer, each 256-byte aligned).
struct DevLayout {
    size_t ops = 0, ops_bytes = 0;       // reference operators (real)
    size_t ops2 = 0, ops2_bytes = 0;     // permuted operators of the FP32 batched kernel
    size_t ops2s = 0, ops2s_bytes = 0;   // tensor-core contexts: the FP32-pipe layout too (ensembles)
    size_t qxy = 0, qxy_bytes = 0;       // FP64 unique-pair schedule: stored metric-averaged operator
    size_t lk = 0, lk_bytes = 0;         // FP64, stored inverse: M^-1 Vh^T per element (lane order)
    size_t gk = 0, gk_bytes = 0;         //   M^-1 Vq^T per element (forcing only)
    size_t pk = 0, pk_bytes = 0;         //   Vh M^-1 Vq^T per element
    size_t vq64 = 0;                     // Vq FP64 (diagnostics)
    size_t geo = 0, wJq = 0, minv = 0, bh = 0, nbr = 0, xq = 0, yq = 0;
    size_t wJq64 = 0, bq64 = 0;
    size_t iwJ = 0;                      // DG-SBP FP64: 1 / (w J) at the nodes
    size_t fmap = 0;                     // DG-SBP: volume node of each face node (int)
    size_t u = 0, res = 0, rhs = 0, ut0 = 0, ut1 = 0;
    size_t partial = 0, diag = 0, status = 0;
    size_t total = 0;
};

struct esdg_ctx {
    esdg_config cfg;
    RefOps ref;
    MeshData mesh;
    std::vector<double> b_modal;  // [K][Np]
    std::vector<unsigned char> image;  // host image of the device layout up to the end of u
    bool prepared = false;             // image holds bathymetry and initial state (esdg_prepare)
    std::string err;
    // device
    bool attached = false;
    bool owns_buffer = false;
    unsigned char* dbuf = nullptr;
    cudaStream_t stream = nullptr;
    DevLayout L;
    LaunchGeom lg;       // k_stage (FP64)
    LaunchGeom lg_proj;  // k_project
    LaunchGeom lg2;      // k_stage2 (FP32)
    int Kpad = 0;        // per-element arrays are padded to a multiple of 8 elements
    int mstride = 0;     // element stride of the packed inverse mass matrices
    bool sbp = false;    // the DG-SBP scheme of Sec. 3 (nodal unknowns at the SBP rule's nodes)
    int ndof = 0;        // unknowns per element and field: Np (modal) or Nq (DG-SBP)
    int nrec = 0;        // node records per element: Nh (hybrid nodes) or Nq (DG-SBP)
    int entropy_parts = 0;
    int num_sms = 0;
    int cur = 0;            // which u~ buffer holds the current stage's values
    bool ut_valid = false;  // u~ buffer current for the state u
    // element partition of one solve (esdg_build_partition); px = py = 1: the whole mesh
    int px = 1, py = 1, part = 0;
    int K_global = 0;
    std::vector<int> owned_gid;  // [K]  global element of each local element
    std::vector<int> ghost_gid;  // [G]  global element of each ghost record (u~ record Kpad + g)
    std::vector<int> ghost_part; // [G]  the part that owns it (ghosts sorted by part, then element)
};

static thread_local std::string g_build_error;

static int fail(esdg_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg; else g_build_error = msg;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                         \
    do {                                                                                            \
        cudaError_t e__ = (call);                                                                   \
        if (e__ != cudaSuccess)                                                                     \
            return fail((ctx), ESDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__));   \
    } while (0)

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t real_size(const esdg_ctx* c) { return c->cfg.precision == ESDG_FP32 ? 4 : 8; }

static int c2_ops_floats(int N);

static bool weight_adjusted(const esdg_config& cfg) { return cfg.mass == ESDG_MASS_WEIGHT_ADJUSTED; }
static bool is_sbp(const esdg_config& cfg) { return cfg.method == ESDG_METHOD_SBP; }
// The FP64 modal path with the stored inverse keeps the inverse's products
// with the shared operators per element, where the kernel's lane mapping
// covers them (two half-warps of modes, one lane per hybrid node): two
// inverse-mass passes and two contractions fewer per stage on the FP64 pipe,
// for 8 (Nh + 1) / 2 * 32 + 8 Nq * 32 bytes per element.
static bool composed_ops(const esdg_config& cfg, const RefOps& R) {
    return cfg.precision == ESDG_FP64 && !is_sbp(cfg) && !weight_adjusted(cfg) && R.Np <= 16 && R.Nh <= 32;
}

// Kernel template parameter of a configuration: NR = N + 8 * rule + 16 * wadg.
static int kernel_nr(const esdg_config& cfg) {
    return cfg.N + (cfg.volume_rule == ESDG_RULE_SYMMETRIC ? 8 : 0) + (weight_adjusted(cfg) ? 16 : 0);
}
// ESDG_DENSE_AUTO: the FP32 pipes, measured faster than the tensor-core form
// at every degree where both exist (the tensor-core form waits on five MMA
// round trips per batch of four elements)
#ifndef ESDG_DENSE_AUTO_TENSOR
#define ESDG_DENSE_AUTO_TENSOR 0
#endif
// The tensor-core form of the FP32 stage kernel exists where Np <= 16 and
// Nq <= 16 (one 16-column MMA round for the lift, Vq and Vq^T).
static bool tc_available(const esdg_config& cfg) {
    return cfg.precision == ESDG_FP32 && cfg.method == ESDG_METHOD_MODAL && !weight_adjusted(cfg) &&
           (cfg.volume_rule == ESDG_RULE_SYMMETRIC ? cfg.N <= 4 : cfg.N <= 3);
}
static bool use_tc(const esdg_config& cfg) {
    if (!tc_available(cfg)) return false;
    return cfg.dense == ESDG_DENSE_TENSOR || (cfg.dense == ESDG_DENSE_AUTO && ESDG_DENSE_AUTO_TENSOR);
}
// template parameter of the FP32 stage kernel: kernel_nr + 32 for the tensor-core form
static int stage2_nr(const esdg_config& cfg) { return kernel_nr(cfg) + (use_tc(cfg) ? 32 : 0); }
#define ESDG_FOR_EACH_NR(X)                                                         \
    X(1) X(2) X(3) X(4) X(5) X(9) X(10) X(11) X(12) X(13) X(17) X(18) X(19) X(20) X(21) \
    X(25) X(26) X(27) X(28) X(29)
// the FP32 stage kernel's template parameters: the above and the tensor-core forms
#define ESDG_FOR_EACH_NR2(X) ESDG_FOR_EACH_NR(X) X(33) X(34) X(35) X(41) X(42) X(43) X(44)

static int pair_steps(int NR);
static int c2_ops_floats(int NR);

static void compute_layout(esdg_ctx* c) {
    const RefOps& R = c->ref;
    const size_t rs = real_size(c);
    const size_t K = size_t(c->mesh.K);
    c->Kpad = int((K + 7) / 8 * 8);
    const size_t Kp = size_t(c->Kpad);
    const int NpP = R.Np * (R.Np + 1) / 2;
    c->mstride = (NpP + 3) & ~3;
    const bool sbp = is_sbp(c->cfg);
    c->sbp = sbp;
    c->ndof = sbp ? R.Nq : R.Np;
    c->nrec = sbp ? R.Nq : R.Nh;
    const size_t nrec = size_t(c->nrec), ndof = size_t(c->ndof);
    DevLayout& L = c->L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.ops_bytes = sbp ? rs * (size_t(R.Nq) * R.Nq * 2 + 3 * size_t(R.Nfq))
                      : rs * (size_t(R.Nh) * R.Nh * 2 + 2 * size_t(R.Nq) * R.Np + 2 * size_t(R.Nh) * R.Np +
                              3 * size_t(R.Nfq) + size_t(R.Nq));
    L.ops = take(L.ops_bytes);
    L.ops2_bytes = c->cfg.precision != ESDG_FP32 ? 0
                   : sbp ? 4 * size_t(sbp2_ops_floats(c->cfg.N))
                         : 4 * size_t(c2_ops_floats(stage2_nr(c->cfg)));
    L.ops2 = take(L.ops2_bytes);
    L.ops2s_bytes = use_tc(c->cfg) ? 4 * size_t(c2_ops_floats(kernel_nr(c->cfg))) : 0;
    L.ops2s = take(L.ops2s_bytes);
    L.vq64 = take(sbp ? 0 : 8 * size_t(R.Nq) * R.Np);
    L.geo = take(rs * Kp * nrec * 4);
    L.wJq = take(rs * Kp * R.Nq);
    L.iwJ = take(sbp && c->cfg.precision == ESDG_FP64 ? 8 * Kp * R.Nq : 0);
    // no stored inverses with the weight-adjusted inverse or the diagonal SBP mass
    L.minv = take((sbp || weight_adjusted(c->cfg)) ? 0 : rs * Kp * c->mstride);
    L.bh = take(rs * Kp * nrec);
    // FP64: the stored metric-averaged operator of the pair schedule (modal:
    // the unique-pair steps; DG-SBP: the Nq x Nq ordered pairs in 32 pieces)
    L.qxy_bytes = c->cfg.precision != ESDG_FP64 ? 0
                  : sbp ? 8 * Kp * size_t((R.Nq * R.Nq + 31) / 32) * 64
                        : 8 * Kp * size_t(pair_steps(kernel_nr(c->cfg))) * 64;
    L.qxy = take(L.qxy_bytes);
    const bool comp = composed_ops(c->cfg, R);
    L.lk_bytes = comp ? 8 * Kp * size_t((R.Nh + 1) / 2) * 32 : 0;
    L.gk_bytes = comp && c->cfg.forcing != ESDG_FORCING_NONE ? 8 * Kp * size_t((R.Nq + 1) / 2) * 32 : 0;
    L.pk_bytes = comp ? 8 * Kp * size_t(R.Nq) * 32 : 0;
    L.lk = take(L.lk_bytes);
    L.gk = take(L.gk_bytes);
    L.pk = take(L.pk_bytes);
    L.nbr = take(4 * Kp * 3);
    L.fmap = take(sbp ? 4 * size_t(R.Nfq) : 0);
    const bool forcing = c->cfg.forcing != ESDG_FORCING_NONE;
    L.xq = take(forcing ? rs * Kp * R.Nq : 0);
    L.yq = take(forcing ? rs * Kp * R.Nq : 0);
    L.wJq64 = take(8 * K * R.Nq);
    L.bq64 = take(8 * K * R.Nq);
    L.u = take(8 * 3 * K * ndof);
    L.res = take(8 * 3 * K * ndof);
    L.rhs = take(8 * 3 * K * ndof);
    // u~ records of the local elements, then one per ghost element of a
    // partition (written by the halo exchange, read as exterior values)
    const size_t Kr = Kp + c->ghost_gid.size();
    L.ut0 = take(rs * Kr * nrec * 4);
    L.ut1 = take(rs * Kr * nrec * 4);
    c->entropy_parts = 1024;
    L.partial = take(8 * 3 * size_t(c->entropy_parts));
    L.diag = take(8 * 4);
    L.status = take(4 * 4);
    L.total = off;
}

template <typename real>
static std::vector<real> to_real(const std::vector<double>& v) {
    return std::vector<real>(v.begin(), v.end());
}

template <typename real>
static std::vector<real> pack_ops(const RefOps& R) {
    // order must match Smem<N, real>: QsT, Vq, VqT, Vh, VhT, wf, nrs, wq
    std::vector<real> o;
    o.reserve(size_t(R.Nh) * R.Nh * 2 + 4 * size_t(R.Nh) * R.Np);
    for (int m = 0; m < R.Nh; ++m)
        for (int l = 0; l < R.Nh; ++l) {
            o.push_back((real)R.Qsr(l, m));
            o.push_back((real)R.Qss(l, m));
        }
    for (int q = 0; q < R.Nq; ++q)
        for (int n = 0; n < R.Np; ++n) o.push_back((real)R.Vq(q, n));
    for (int n = 0; n < R.Np; ++n)
        for (int q = 0; q < R.Nq; ++q) o.push_back((real)R.Vq(q, n));
    for (int l = 0; l < R.Nh; ++l)
        for (int n = 0; n < R.Np; ++n) o.push_back((real)R.Vh(l, n));
    for (int n = 0; n < R.Np; ++n)
        for (int l = 0; l < R.Nh; ++l) o.push_back((real)R.Vh(l, n));
    for (int f = 0; f < R.Nfq; ++f) o.push_back((real)R.wf[f]);
    for (int f = 0; f < R.Nfq; ++f) {
        o.push_back((real)R.nr[f]);
        o.push_back((real)R.ns[f]);
    }
    for (int q = 0; q < R.Nq; ++q) o.push_back((real)R.wq[q]);
    return o;
}

// Operators of the DG-SBP kernel (SbpSmem in esdg_sbp.cuh): the skew SBP
// operators Q_SBP - Q_SBP^T = [I; I_f]^T (Q_h - Q_h^T) [I; I_f] (Theorem 3.1)
// as [Nq(m)][Nq(l)][2] = (r, s) pairs, then w_f and the scaled normals.
template <typename real>
static std::vector<real> pack_ops_sbp(const RefOps& R) {
    const int Nq = R.Nq;
    auto node = [&](int a) { return a < Nq ? a : R.fmap[a - Nq]; };
    Mat Sr(Nq, Nq), Ss(Nq, Nq);
    for (int a = 0; a < R.Nh; ++a)
        for (int b = 0; b < R.Nh; ++b) {
            Sr(node(a), node(b)) += R.Qsr(a, b);
            Ss(node(a), node(b)) += R.Qss(a, b);
        }
    std::vector<real> o;
    o.reserve(size_t(Nq) * Nq * 2 + 3 * size_t(R.Nfq));
    for (int m = 0; m < Nq; ++m)
        for (int l = 0; l < Nq; ++l) {
            o.push_back((real)Sr(l, m));
            o.push_back((real)Ss(l, m));
        }
    for (int f = 0; f < R.Nfq; ++f) o.push_back((real)R.wf[f]);
    for (int f = 0; f < R.Nfq; ++f) {
        o.push_back((real)R.nr[f]);
        o.push_back((real)R.ns[f]);
    }
    return o;
}

// Operators of the FP32 batched DG-SBP kernel in its shared-memory layout (S2<N>
// in esdg_sbp2.cuh): the skew SBP operators / 8 per (column, lane slot), w_f,
// the scaled normals, and the face-node / volume-node maps as int bits.
template <int N>
static std::vector<float> pack_ops_sbp2_t(const RefOps& R) {
    typedef S2<N> C;
    const int Nq = R.Nq, LPE = C::LPE;
    const std::vector<double> full = pack_ops_sbp<double>(R);  // [m][l][2], then w_f, normals
    std::vector<float> o(C::o_end, 0.f);
    for (int m = 0; m < Nq; ++m)
        for (int b = 0; b < LPE; ++b)
            for (int i = 0; i < C::RPL; ++i) {
                const int l = b + LPE * i;
                if (l >= Nq) continue;
                o[C::o_Qs + (m * LPE + b) * C::OPB + 2 * i] = (float)(0.125 * full[(size_t(m) * Nq + l) * 2]);
                o[C::o_Qs + (m * LPE + b) * C::OPB + 2 * i + 1] = (float)(0.125 * full[(size_t(m) * Nq + l) * 2 + 1]);
            }
    const size_t base = size_t(Nq) * Nq * 2;
    for (int f = 0; f < R.Nfq; ++f) {
        o[C::o_wf + f] = (float)full[base + f];
        o[C::o_nrs + 2 * f] = (float)full[base + R.Nfq + 2 * f];
        o[C::o_nrs + 2 * f + 1] = (float)full[base + R.Nfq + 2 * f + 1];
    }
    std::vector<int> frow(Nq, -1);
    for (int f = 0; f < R.Nfq; ++f) frow[R.fmap[f]] = f;
    std::memcpy(o.data() + C::o_fmap, R.fmap.data(), sizeof(int) * R.Nfq);
    std::memcpy(o.data() + C::o_frow, frow.data(), sizeof(int) * Nq);
    return o;
}

static std::vector<float> pack_ops_sbp2(const RefOps& R) {
    switch (R.N) {
        case 1: return pack_ops_sbp2_t<1>(R);
        case 2: return pack_ops_sbp2_t<2>(R);
        case 3: return pack_ops_sbp2_t<3>(R);
        case 4: return pack_ops_sbp2_t<4>(R);
        case 5: return pack_ops_sbp2_t<5>(R);
    }
    return {};
}

// TF32 rounding (to nearest, ties to even) of a finite float.
static float tf32_round(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x0FFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
    std::memcpy(&f, &u, 4);
    return f;
}

// One B operand block of the tensor-core contractions: rows x K entries
// op(n, k) (zero outside nr x nk), as the TF32 pair (hi at o + base, lo at
// o + base + rows K), entry (n, k) at (n / 8) 8 K + (k / 4) 32 + (n % 8) 4 + k % 4.
template <typename F>
static void put_tc_block(std::vector<float>& o, int base, int rows, int K, int nr, int nk, F op) {
    for (int n = 0; n < rows; ++n)
        for (int k = 0; k < K; ++k) {
            const double v = (n < nr && k < nk) ? op(n, k) : 0.0;
            const float hi = tf32_round((float)v);
            const float lo = tf32_round((float)(v - (double)hi));
            const int i = (n / 8) * 8 * K + (k / 4) * 32 + (n % 8) * 4 + k % 4;
            o[base + i] = hi;
            o[base + rows * K + i] = lo;
        }
}

// Operators of k_stage2 in its shared-memory layout (see C2<N> in esdg_stage2.cuh).
template <int N>
static std::vector<float> pack_ops2_t(const RefOps& R) {
    typedef C2<N> C;
    const int LPE = C::LPE;
    std::vector<float> o(C::o_end, 0.f);
    if (C::UP) {
        // unique pairs: entries (Qr, Qs) of own volume row l = b + LPE i
        // against partner row m = (b + s) mod LPE + LPE j, in the order of
        // the kernel's offset schedule; zero where the pair is not this
        // lane's (offset LPE/2 of the volume-volume block: lanes b < LPE/2
        // take (i, j) = (0, 0), (1, 1), the others (0, 1), (1, 0)) or m >= Nh
        auto put4 = [&](int at, int b, int s, int j, bool half) {
            const int m = ((b + s) % LPE) + LPE * j;
            for (int i = 0; i < C::VS; ++i) {
                const int l = b + LPE * i;
                bool take = m < R.Nh;
                if (half) take = take && ((b < LPE / 2) == (i == j));
                o[at + 4 * b + 2 * i] = take ? (float)R.Qsr(l, m) : 0.f;
                o[at + 4 * b + 2 * i + 1] = take ? (float)R.Qss(l, m) : 0.f;
            }
        };
        for (int b = 0; b < LPE; ++b) {
            o[C::o_U0 + 2 * b] = (float)R.Qsr(b, b + LPE);
            o[C::o_U0 + 2 * b + 1] = (float)R.Qss(b, b + LPE);
            for (int s = 1; s <= LPE / 2; ++s)
                for (int j = 0; j < C::VS; ++j)
                    put4(C::o_Uvv + ((s - 1) * C::VS + j) * LPE * 4, b, s, j, s == LPE / 2);
            for (int s = 0; s < LPE; ++s)
                for (int j = C::VS; j < C::RPL; ++j)
                    put4(C::o_Uvf + (s * C::FS + (j - C::VS)) * LPE * 4, b, s, j, false);
        }
    } else {
        for (int m = 0; m < R.Nh; ++m)
            for (int b = 0; b < LPE; ++b)
                for (int i = 0; i < C::RPL; ++i) {
                    const int l = b + LPE * i;
                    if (l >= R.Nh) continue;
                    o[C::o_Qs + (m * LPE + b) * C::OPB + 2 * i] = (float)R.Qsr(l, m);
                    o[C::o_Qs + (m * LPE + b) * C::OPB + 2 * i + 1] = (float)R.Qss(l, m);
                }
    }
    if (C::TC) {
        // lift Vh^T, Vq, Vq^T, Vh as tensor-core B operands (rows = outputs, K = inputs)
        const int t = C::o_tc;
        put_tc_block(o, t + C::tb_lift, C::NpR, C::KL, R.Np, R.Nh, [&](int n, int l) { return R.Vh(l, n); });
        put_tc_block(o, t + C::tb_vq, C::NqR, C::KM, R.Nq, R.Np, [&](int q, int n) { return R.Vq(q, n); });
        put_tc_block(o, t + C::tb_vqt, C::NpR, C::KQ, R.Np, R.Nq, [&](int n, int q) { return R.Vq(q, n); });
        put_tc_block(o, t + C::tb_vh, C::NhR, C::KM, R.Nh, R.Np, [&](int l, int n) { return R.Vh(l, n); });
    }
    if (!C::WADG && !C::TC)
        for (int l = 0; l < R.Nh; ++l)
            for (int b = 0; b < LPE; ++b)
                for (int j = 0; j < C::MPL; ++j) {
                    const int n = b + LPE * j;
                    if (n < R.Np) o[C::o_VhT + (l * LPE + b) * C::MPLp + j] = (float)R.Vh(l, n);
                }
    if (!C::TC)
    for (int q = 0; q < R.Nq; ++q)
        for (int b = 0; b < LPE; ++b)
            for (int j = 0; j < C::MPL; ++j) {
                const int n = b + LPE * j;
                if (n < R.Np) o[C::o_VqT + (q * LPE + b) * C::MPLp + j] = (float)R.Vq(q, n);
            }
    if (!C::TC)
    for (int n = 0; n < R.Np; ++n)
        for (int b = 0; b < LPE; ++b) {
            for (int j = 0; j < C::QPL; ++j) {
                const int q = b + LPE * j;
                if (q < R.Nq) o[C::o_Vq + (n * LPE + b) * C::QPLp + j] = (float)R.Vq(q, n);
            }
            for (int j = 0; j < C::RPL; ++j) {
                const int l = b + LPE * j;
                if (!C::WADG && l < R.Nh) o[C::o_Vh + (n * LPE + b) * C::RPLp + j] = (float)R.Vh(l, n);
            }
        }
    if (C::WADG) {
        // composed factors of the weight-adjusted inverse, formed in FP64:
        // C = Vq Vh^T (Nq x Nh), A = Vq Vq^T (Nq x Nq), B = Vh Vq^T (Nh x Nq)
        const Mat Cm = matmul(R.Vq, transpose(R.Vh)), Am = matmul(R.Vq, transpose(R.Vq)), Bm = transpose(Cm);
        for (int b = 0; b < LPE; ++b) {
            for (int j = 0; j < C::QPL; ++j) {
                const int q = b + LPE * j;
                if (q >= R.Nq) continue;
                for (int l = 0; l < R.Nh; ++l) o[C::o_C + (l * LPE + b) * C::QPLp + j] = (float)Cm(q, l);
                for (int q2 = 0; q2 < R.Nq; ++q2) o[C::o_A + (q2 * LPE + b) * C::QPLp + j] = (float)Am(q, q2);
            }
            for (int j = 0; j < C::RPL; ++j) {
                const int l = b + LPE * j;
                if (l >= R.Nh) continue;
                for (int q = 0; q < R.Nq; ++q) o[C::o_B + (q * LPE + b) * C::RPLp + j] = (float)Bm(l, q);
            }
        }
        for (int q = 0; q < R.Nq; ++q) o[C::o_wq + q] = (float)R.wq[q];
    }
    for (int f = 0; f < R.Nfq; ++f) {
        o[C::o_wf + f] = (float)R.wf[f];
        o[C::o_nrs + 2 * f] = (float)R.nr[f];
        o[C::o_nrs + 2 * f + 1] = (float)R.ns[f];
    }
    return o;
}

static int c2_ops_floats(int NR) {
    switch (NR) {
#define X(v) case v: return C2<v>::o_end;
        ESDG_FOR_EACH_NR2(X)
#undef X
    }
    return 0;
}

static std::vector<float> pack_ops2(const RefOps& R, int NR) {
    switch (NR) {
#define X(v) case v: return pack_ops2_t<v>(R);
        ESDG_FOR_EACH_NR2(X)
#undef X
    }
    return {};
}

// ---- host image of the device layout ------------------------------------------
// Everything up to the end of the state u is built in host memory (operators,
// geometry, bathymetry, initial state) and reaches the device in one copy.
template <typename T>
static void put(std::vector<unsigned char>& img, size_t off, const std::vector<T>& v) {
    std::memcpy(img.data() + off, v.data(), v.size() * sizeof(T));
}

// The FP64 kernel's unique-pair schedule (PairSched in esdg_kernels.cuh):
// steps per element, 0 where the rule is too large for it.
static int pair_steps(int NR) {
    switch (NR) {
#define X(v) case v: return PairSched<v>::SPLIT ? PairSched<v>::NSTEP : 0;
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return 0;
}

// The metric-averaged skew operator entries the FP64 kernel's lanes take,
// element by element and step by step: lane (half-warp hf, row j) of step s
// pairs volume row j with column m (the kernel's diagonal schedule) and holds
// Qx = q_r (rx_j + rx_m) + q_s (sx_j + sx_m), Qy likewise with ry, sy, where
// (q_r, q_s) = (Qskew^r, Qskew^s)[j][m] and the metrics are the kernel's own
// (geo, [K][Nh][4], scaled by 1/8 as the kernel scales them); zero where the
// lane has no pair.  Stage-independent.
template <int NR>
static std::vector<double> pair_operator_t(const esdg_ctx* c, const std::vector<double>& geo) {
    typedef PairSched<NR> PS;
    const RefOps& R = c->ref;
    const int Nh = R.Nh, K = c->mesh.K;
    std::vector<double> q(size_t(c->Kpad) * PS::NSTEP * 64, 0.0);
    if (!PS::SPLIT) return q;
    for (int e = 0; e < K; ++e) {
        const double* g = geo.data() + size_t(e) * Nh * 4;
        for (int st = 0; st < PS::NSTEP; ++st)
            for (int lane = 0; lane < 32; ++lane) {
                const int j = lane & 15, hf = lane >> 4;
                int m = -1;
                if (st < PS::SVV0) {
                    const int d = hf == 0 ? 1 + st : PS::SVV0 + 1 + st;
                    if (j < PS::V && d <= PS::SVV && !(2 * d == PS::V && j >= PS::V / 2)) m = (j + d) % PS::V;
                } else {
                    const int k = st - PS::SVV0;
                    const int t = hf == 0 ? k : PS::SVF0 + k;
                    const int f = (j + t) % PS::L;
                    if (j < PS::V && t < PS::L && f < PS::F) m = PS::V + f;
                }
                if (m < 0) continue;
                const double qr = R.Qsr(j, m), qs = R.Qss(j, m);
                const double* gj = g + 4 * j;
                const double* gm = g + 4 * m;
                double* o = q.data() + ((size_t(e) * PS::NSTEP + st) * 32 + lane) * 2;
                // the kernel carries the metrics scaled by 1/8 (exact)
                o[0] = qr * (0.125 * gj[0] + 0.125 * gm[0]) + qs * (0.125 * gj[1] + 0.125 * gm[1]);
                o[1] = qr * (0.125 * gj[2] + 0.125 * gm[2]) + qs * (0.125 * gj[3] + 0.125 * gm[3]);
            }
    }
    return q;
}

// The same for the DG-SBP FP64 kernel, whose lanes take the Nq x Nq ordered
// pairs (l, m), row-major, in 32 pieces of PL = ceil(Nq^2 / 32): entry it of
// lane i is pair i PL + it, laid out [K][PL][32][2]; qsbp is the packed SBP
// skew operator ([m][l][2]) and geo the metrics at the SBP nodes ([K][Nq][4]).
template <typename real>
static std::vector<double> sbp_pair_operator(const esdg_ctx* c, const std::vector<double>& qsbp,
                                             const std::vector<real>& geo) {
    const int Nq = c->ref.Nq, K = c->mesh.K;
    const int PL = (Nq * Nq + 31) / 32;
    std::vector<double> q(size_t(c->Kpad) * PL * 64, 0.0);
    for (int e = 0; e < K; ++e) {
        const real* g = geo.data() + size_t(e) * Nq * 4;
        for (int lane = 0; lane < 32; ++lane)
            for (int it = 0; it < PL; ++it) {
                const int pp = lane * PL + it;
                if (pp >= Nq * Nq) continue;
                const int r = pp / Nq, m = pp - r * Nq;
                const double qr = qsbp[(size_t(m) * Nq + r) * 2], qs = qsbp[(size_t(m) * Nq + r) * 2 + 1];
                const real* gr = g + 4 * r;
                const real* gm = g + 4 * m;
                double* o = q.data() + ((size_t(e) * PL + it) * 32 + lane) * 2;
                o[0] = qr * (0.125 * gr[0] + 0.125 * gm[0]) + qs * (0.125 * gr[1] + 0.125 * gm[1]);
                o[1] = qr * (0.125 * gr[2] + 0.125 * gm[2]) + qs * (0.125 * gr[3] + 0.125 * gm[3]);
            }
    }
    return q;
}

template <typename real>
static std::vector<double> pair_operator(const esdg_ctx* c, const std::vector<real>& geo) {
    std::vector<double> g(geo.begin(), geo.end());
    switch (kernel_nr(c->cfg)) {
#define X(v) case v: return pair_operator_t<v>(c, g);
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return {};
}

static void composed_operators(const esdg_ctx* c, std::vector<unsigned char>& img);

template <typename real>
static void fill_static(const esdg_ctx* c, std::vector<unsigned char>& img) {
    const RefOps& R = c->ref;
    const MeshData& M = c->mesh;
    const size_t K = size_t(M.K);
    if (c->sbp) {
        put(img, c->L.ops, pack_ops_sbp<real>(R));
        put(img, c->L.fmap, R.fmap);
        if (c->cfg.precision == ESDG_FP32) put(img, c->L.ops2, pack_ops_sbp2(R));
        // metrics at the SBP nodes (the volume part of the hybrid nodes)
        std::vector<real> geo(K * R.Nq * 4);
        for (size_t e = 0; e < K; ++e)
            for (size_t i = 0; i < size_t(R.Nq) * 4; ++i) geo[e * R.Nq * 4 + i] = (real)M.geo[e * R.Nh * 4 + i];
        put(img, c->L.geo, geo);
        if (c->L.qxy_bytes) put(img, c->L.qxy, sbp_pair_operator(c, pack_ops_sbp<double>(R), geo));
    } else {
        put(img, c->L.ops, pack_ops<real>(R));
        put(img, c->L.vq64, R.Vq.a);
        // the FP32 batched kernel reads the metrics pre-scaled by 1/8 (exact)
        const double gscale = c->cfg.precision == ESDG_FP32 ? 0.125 : 1.0;
        std::vector<real> geo(M.geo.size());
        for (size_t i = 0; i < geo.size(); ++i) geo[i] = (real)(gscale * M.geo[i]);
        put(img, c->L.geo, geo);
        if (c->L.qxy_bytes) put(img, c->L.qxy, pair_operator(c, geo));
        if (c->cfg.precision == ESDG_FP32) put(img, c->L.ops2, pack_ops2(R, stage2_nr(c->cfg)));
        if (use_tc(c->cfg)) put(img, c->L.ops2s, pack_ops2(R, kernel_nr(c->cfg)));
    }
    std::vector<double> wJ64(K * R.Nq);
    for (size_t e = 0; e < K; ++e)
        for (int q = 0; q < R.Nq; ++q) wJ64[e * R.Nq + q] = R.wq[q] * M.Jq[e * R.Nq + q];
    put(img, c->L.wJq, to_real<real>(wJ64));
    put(img, c->L.wJq64, wJ64);
    if (c->sbp && c->cfg.precision == ESDG_FP64) {
        std::vector<double> iw(wJ64.size());
        for (size_t i = 0; i < iw.size(); ++i) iw[i] = 1.0 / wJ64[i];
        put(img, c->L.iwJ, iw);
    }
    if (!weight_adjusted(c->cfg) && !c->sbp) {
        const int NpP = R.Np * (R.Np + 1) / 2;
        std::vector<real> mi(K * size_t(c->mstride), (real)0);
        for (size_t e = 0; e < K; ++e)
            for (int i = 0; i < NpP; ++i) mi[e * c->mstride + i] = (real)M.minv[e * NpP + i];
        put(img, c->L.minv, mi);
    }
    if (c->L.lk_bytes) composed_operators(c, img);
    put(img, c->L.nbr, M.nbr);
    if (c->cfg.forcing != ESDG_FORCING_NONE) {
        put(img, c->L.xq, to_real<real>(M.xq));
        put(img, c->L.yq, to_real<real>(M.yq));
    }
}

// b at the hybrid nodes (real) and at the volume nodes (FP64) from b_modal.
template <typename real>
static void bathymetry_arrays(const esdg_ctx* c, std::vector<real>& bhr, std::vector<double>& bq) {
    const RefOps& R = c->ref;
    const size_t K = size_t(c->mesh.K);
    const int nrec = c->nrec;  // hybrid nodes, or the SBP nodes (the first Nq rows of V_h)
    bhr.assign(K * nrec, (real)0);
    bq.assign(K * R.Nq, 0.0);
    for (size_t e = 0; e < K; ++e)
        for (int l = 0; l < nrec; ++l) {
            double s = 0;
            for (int n = 0; n < R.Np; ++n) s += R.Vh(l, n) * c->b_modal[e * R.Np + n];
            bhr[e * nrec + l] = (real)s;
            if (l < R.Nq) bq[e * R.Nq + l] = s;
        }
}

// J-weighted L2 projection of q (at volume points) onto the modes; SURFACE
// mode takes q[0] = H and subtracts the modal bathymetry.
static void project_host(const esdg_ctx* c, const double* q_volq, int mode, double* u) {
    const RefOps& R = c->ref;
    const MeshData& M = c->mesh;
    const size_t K = size_t(M.K);
    if (c->sbp) {
        // DG-SBP: the unknowns are the nodal values themselves (SURFACE: h = H - b)
        for (int f = 0; f < 3; ++f)
            for (size_t e = 0; e < K; ++e)
                for (int q = 0; q < R.Nq; ++q) {
                    double v = q_volq[(f * K + e) * R.Nq + q];
                    if (f == 0 && mode == ESDG_INIT_SURFACE)
                        for (int n = 0; n < R.Np; ++n) v -= R.Vq(q, n) * c->b_modal[e * R.Np + n];
                    u[(f * K + e) * R.Nq + q] = v;
                }
        return;
    }
    const int NpP = R.Np * (R.Np + 1) / 2;
    std::vector<double> y(R.Np);
    for (int f = 0; f < 3; ++f)
        for (size_t e = 0; e < K; ++e) {
            for (int n = 0; n < R.Np; ++n) {
                double s = 0;
                for (int q = 0; q < R.Nq; ++q)
                    s += R.Vq(q, n) * R.wq[q] * M.Jq[e * R.Nq + q] * q_volq[(f * K + e) * R.Nq + q];
                y[n] = s;
            }
            const double* mi = &M.minv[e * NpP];
            for (int n = 0; n < R.Np; ++n) {
                double s = 0;
                for (int j = 0; j < R.Np; ++j) s += mi[n >= j ? n * (n + 1) / 2 + j : j * (j + 1) / 2 + n] * y[j];
                if (f == 0 && mode == ESDG_INIT_SURFACE) s -= c->b_modal[e * R.Np + n];
                u[(f * K + e) * R.Np + n] = s;
            }
        }
}

static void modal_bathymetry(esdg_ctx* c, const double* b_nodal) {
    const RefOps& R = c->ref;
    const size_t K = size_t(c->mesh.K);
    for (size_t e = 0; e < K; ++e)
        for (int n = 0; n < R.Np; ++n) {
            double s = 0;
            for (int m = 0; m < R.Np; ++m) s += R.Veq_inv(n, m) * b_nodal[e * R.Np + m];
            c->b_modal[e * R.Np + n] = s;
        }
}

// Per-element products of the FP64 path (composed_ops): L = M^-1 Vh^T,
// G = M^-1 Vq^T and P = Vh G, formed in FP64 from the element's inverse mass
// and written into the image in the lanes' order of k_stage / project_element.
static void composed_operators(const esdg_ctx* c, std::vector<unsigned char>& img) {
    const RefOps& R = c->ref;
    const MeshData& M = c->mesh;
    const int K = M.K, Np = R.Np, Nq = R.Nq, Nh = R.Nh, LT = (Nh + 1) / 2, GT = (Nq + 1) / 2;
    double* lk = reinterpret_cast<double*>(img.data() + c->L.lk);
    double* gk = c->L.gk_bytes ? reinterpret_cast<double*>(img.data() + c->L.gk) : nullptr;
    double* pk = reinterpret_cast<double*>(img.data() + c->L.pk);
    std::memset(lk, 0, c->L.lk_bytes);
    std::memset(pk, 0, c->L.pk_bytes);
    if (gk) std::memset(gk, 0, c->L.gk_bytes);
    auto work = [&](int e0, int e1) {
        std::vector<double> mi(size_t(Np) * Np), G(size_t(Np) * Nq), Lm(size_t(Np) * Nh);
        for (int e = e0; e < e1; ++e) {
            const double* pm = &M.minv[size_t(e) * Np * (Np + 1) / 2];
            for (int n = 0; n < Np; ++n)
                for (int j = 0; j < Np; ++j) mi[n * Np + j] = pm[n >= j ? n * (n + 1) / 2 + j : j * (j + 1) / 2 + n];
            for (int n = 0; n < Np; ++n) {
                for (int q = 0; q < Nq; ++q) {
                    double s = 0;
                    for (int j = 0; j < Np; ++j) s += mi[n * Np + j] * R.Vq(q, j);
                    G[n * Nq + q] = s;
                }
                for (int l = 0; l < Nh; ++l) {
                    double s = 0;
                    for (int j = 0; j < Np; ++j) s += mi[n * Np + j] * R.Vh(l, j);
                    Lm[n * Nh + l] = s;
                }
            }
            // lane n + 16 hf, step t: column hf * LT + t (L) or hf * GT + t (G)
            for (int lane = 0; lane < 32; ++lane) {
                const int n = lane & 15, hf = lane >> 4;
                if (n >= Np) continue;
                for (int t = 0; t < LT; ++t) {
                    const int l = hf * LT + t;
                    if (l < Nh) lk[(size_t(e) * LT + t) * 32 + lane] = Lm[n * Nh + l];
                }
                if (gk)
                    for (int t = 0; t < GT; ++t) {
                        const int q = hf * GT + t;
                        if (q < Nq) gk[(size_t(e) * GT + t) * 32 + lane] = G[n * Nq + q];
                    }
            }
            for (int l = 0; l < Nh; ++l)
                for (int q = 0; q < Nq; ++q) {
                    double s = 0;
                    for (int n = 0; n < Np; ++n) s += R.Vh(l, n) * G[n * Nq + q];
                    pk[(size_t(e) * Nq + q) * 32 + l] = s;
                }
        }
    };
    const int nt = std::max(1, std::min<int>(16, std::min<int>(int(std::thread::hardware_concurrency()),
                                                                (K + 1023) / 1024)));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(work, int(size_t(K) * t / nt), int(size_t(K) * (t + 1) / nt));
    work(0, K / nt);
    for (auto& th : pool) th.join();
}

// Host image of [0, end of u): operators, geometry, bathymetry and (if q is
// given) the projected initial state.
template <typename real>
static void build_image(esdg_ctx* c, const double* q_volq, int mode) {
    c->image.assign(c->L.res, 0);
    fill_static<real>(c, c->image);
    std::vector<real> bhr;
    std::vector<double> bq;
    bathymetry_arrays<real>(c, bhr, bq);
    put(c->image, c->L.bh, bhr);
    put(c->image, c->L.bq64, bq);
    if (q_volq) project_host(c, q_volq, mode, reinterpret_cast<double*>(c->image.data() + c->L.u));
}

template <typename real>
static int upload_bathymetry_t(esdg_ctx* c) {
    std::vector<real> bhr;
    std::vector<double> bq;
    bathymetry_arrays<real>(c, bhr, bq);
    CUDA_TRY(c, cudaMemcpyAsync(c->dbuf + c->L.bh, bhr.data(), bhr.size() * sizeof(real), cudaMemcpyHostToDevice,
                                c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->dbuf + c->L.bq64, bq.data(), bq.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->ut_valid = false;
    return ESDG_OK;
}

static int upload_bathymetry(esdg_ctx* c) {
    return c->cfg.precision == ESDG_FP32 ? upload_bathymetry_t<float>(c) : upload_bathymetry_t<double>(c);
}

template <typename real>
static StageParams<real> make_params(esdg_ctx* c) {
    StageParams<real> p;
    std::memset(&p, 0, sizeof(p));
    const RefOps& R = c->ref;
    unsigned char* d = c->dbuf;
    p.K = c->mesh.K;
    p.g = (real)c->cfg.g;
    p.lf = c->cfg.lax_friedrichs;
    real* ops = reinterpret_cast<real*>(d + c->L.ops);
    p.QsT = ops;
    if (c->sbp) {
        p.wf = p.QsT + size_t(R.Nq) * R.Nq * 2;
        p.nrs = p.wf + R.Nfq;
        p.fmap = reinterpret_cast<const int*>(d + c->L.fmap);
    } else {
        p.Vq = p.QsT + size_t(R.Nh) * R.Nh * 2;
        p.VqT = p.Vq + size_t(R.Nq) * R.Np;
        p.Vh = p.VqT + size_t(R.Np) * R.Nq;
        p.VhT = p.Vh + size_t(R.Nh) * R.Np;
        p.wf = p.VhT + size_t(R.Np) * R.Nh;
        p.nrs = p.wf + R.Nfq;
        p.wq = p.nrs + 2 * size_t(R.Nfq);
    }
    p.geo = reinterpret_cast<const real*>(d + c->L.geo);
    p.wJq = reinterpret_cast<const real*>(d + c->L.wJq);
    p.iwJ = (c->sbp && c->cfg.precision == ESDG_FP64) ? reinterpret_cast<const real*>(d + c->L.iwJ) : nullptr;
    p.minv = reinterpret_cast<const real*>(d + c->L.minv);
    p.mstride = c->mstride;
    p.bh = reinterpret_cast<const real*>(d + c->L.bh);
    p.nbr = reinterpret_cast<const int*>(d + c->L.nbr);
    p.walls = c->cfg.boundary == ESDG_BOUNDARY_WALLS;
    p.xq = reinterpret_cast<const real*>(d + c->L.xq);
    p.yq = reinterpret_cast<const real*>(d + c->L.yq);
    p.qxy = reinterpret_cast<const real*>(d + c->L.qxy);
    p.lk = c->L.lk_bytes ? reinterpret_cast<const real*>(d + c->L.lk) : nullptr;
    p.gk = c->L.gk_bytes ? reinterpret_cast<const real*>(d + c->L.gk) : nullptr;
    p.pk = c->L.pk_bytes ? reinterpret_cast<const real*>(d + c->L.pk) : nullptr;
    p.u = reinterpret_cast<double*>(d + c->L.u);
    p.u_in = p.u;
    p.res = reinterpret_cast<double*>(d + c->L.res);
    p.rhs_out = reinterpret_cast<double*>(d + c->L.rhs);
    p.forcing = c->cfg.forcing;
    p.mms_amp = (real)c->cfg.mms_amp;
    p.mms_bamp = (real)c->cfg.mms_bamp;
    p.mms_u0 = (real)c->cfg.mms_u0;
    p.mms_v0 = (real)c->cfg.mms_v0;
    p.status = reinterpret_cast<int*>(d + c->L.status);
    return p;
}

template <typename real>
static real* ut_buf(esdg_ctx* c, int which) {
    return reinterpret_cast<real*>(c->dbuf + (which == 0 ? c->L.ut0 : c->L.ut1));
}

// ---- degree dispatch ---------------------------------------------------------
template <typename real>
static cudaError_t d_sbp(esdg_ctx* c, const StageParams<real>& p, int mode) {
    if constexpr (std::is_same<real, float>::value) {
        // FP32 stages on the batched kernel; record preparation on the generic one
        const float* ops2 = reinterpret_cast<const float*>(c->dbuf + c->L.ops2);
        if (mode != 2) switch (c->cfg.N) {
#define X(v) case v: return launch_sbp2<v>(p, ops2, c->Kpad, mode, c->lg2, c->stream);
            X(1) X(2) X(3) X(4) X(5)
#undef X
        }
    }
    switch (c->cfg.N) {
#define X(v) case v: return launch_sbp<v, real>(p, mode, c->lg, c->stream);
        X(1) X(2) X(3) X(4) X(5)
#undef X
    }
    return cudaErrorInvalidValue;
}

static cudaError_t d_geometry(esdg_ctx* c) {
    const int sms = c->num_sms;
    cudaError_t e = cudaErrorInvalidValue;
    if (c->sbp) {
        const bool f32 = c->cfg.precision == ESDG_FP32;
        switch (c->cfg.N) {
#define X(v)                                                                       \
    case v:                                                                        \
        e = f32 ? sbp_geometry<v, float>(sms, c->lg) : sbp_geometry<v, double>(sms, c->lg); \
        if (!e && f32) e = sbp2_geometry<v>(sms, c->lg2);                          \
        break;
            X(1) X(2) X(3) X(4) X(5)
#undef X
        }
        return e;
    }
    if (c->cfg.precision == ESDG_FP32) {
        switch (stage2_nr(c->cfg)) {
#define X(v) case v: e = stage2_geometry<v>(sms, c->lg2); break;
            ESDG_FOR_EACH_NR2(X)
#undef X
        }
    } else {
        switch (kernel_nr(c->cfg)) {
#define X(v) case v: e = project_geometry<v, double>(sms, c->lg_proj); if (!e) e = stage_geometry<v, double>(sms, c->lg); break;
            ESDG_FOR_EACH_NR(X)
#undef X
        }
    }
    return e;
}
static cudaError_t d_project(int NR, const StageParams<double>& p, const LaunchGeom& lg, cudaStream_t s) {
    switch (NR) {
#define X(v) case v: return launch_project<v, double>(p, lg, s);
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
static cudaError_t d_stage(esdg_ctx* c, const StageParams<double>& p, int mode) {
    if (c->sbp) return d_sbp<double>(c, p, mode);
    const LaunchGeom& lg = c->lg;
    switch (kernel_nr(c->cfg)) {
#define X(v) case v: return launch_stage<v, double>(p, mode, lg, c->stream);
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
static cudaError_t d_stage(esdg_ctx* c, const StageParams<float>& p, int mode) {
    if (c->sbp) return d_sbp<float>(c, p, mode);
    const LaunchGeom& lg = c->lg2;
    const float* ops2 = reinterpret_cast<const float*>(c->dbuf + c->L.ops2);
    switch (stage2_nr(c->cfg)) {
#define X(v) case v: return launch_stage2<v>(p, ops2, c->Kpad, mode, lg, c->stream);
        ESDG_FOR_EACH_NR2(X)
#undef X
    }
    return cudaErrorInvalidValue;
}
static cudaError_t d_entropy(int NR, int K, double g, const double* u, const double* rhs, const double* Vq,
                             const double* wJq, const double* bq, double* partial, int nparts, double* out,
                             cudaStream_t s) {
    switch (NR) {
#define X(v) case v: return launch_entropy<v>(K, g, u, rhs, Vq, wJq, bq, partial, nparts, out, s);
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

static int check_status(esdg_ctx* c) {
    int st[1] = {0};
    int* dst = reinterpret_cast<int*>(c->dbuf + c->L.status);
    CUDA_TRY(c, cudaMemcpyAsync(st, dst, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (st[0]) {
        CUDA_TRY(c, cudaMemsetAsync(dst, 0, 4, c->stream));
        if (st[0] & STATUS_TIMEOUT)
            return fail(c, ESDG_ETIMEOUT, "a bounded wait on an asynchronous copy expired in the stage kernel");
        if (st[0] & STATUS_NONFINITE) return fail(c, ESDG_ENONFINITE, "non-finite entropy-projected state");
        return fail(c, ESDG_ENONPOSITIVE, "non-positive (entropy-projected) depth");
    }
    return ESDG_OK;
}

template <typename real>
static int project_current(esdg_ctx* c, const double* u_in, int target, bool copy_in = false) {
    StageParams<real> p = make_params<real>(c);
    if (u_in) p.u_in = u_in;
    p.copy_in = copy_in ? 1 : 0;  // also store u_in as the state, residual zeroed
    p.ut_out = ut_buf<real>(c, target);
    if constexpr (std::is_same<real, float>::value) {
        CUDA_TRY(c, d_stage(c, p, 2));  // the FP32 path's projection-only stage kernel (or DG-SBP records)
    } else {
        if (c->sbp)
            CUDA_TRY(c, d_stage(c, p, 2));  // DG-SBP: nodal records of the state
        else
            CUDA_TRY(c, d_project(kernel_nr(c->cfg), p, c->lg_proj, c->stream));
    }
    return ESDG_OK;
}

template <typename real>
static int rhs_t(esdg_ctx* c, double t, const double* u_in, double* rhs_out) {
    int rc = project_current<real>(c, u_in, c->cur ^ 1);
    if (rc) return rc;
    StageParams<real> p = make_params<real>(c);
    p.ut_in = ut_buf<real>(c, c->cur ^ 1);
    p.rhs_out = rhs_out;
    p.t = t;
    CUDA_TRY(c, d_stage(c, p, 0));
    return ESDG_OK;
}

// nsteps LSRK45 steps; if u_out is set, the last stage also writes the new
// state there (a host buffer the device can write).
template <typename real>
static int step_t(esdg_ctx* c, int nsteps, double dt, double t0, double* u_out = nullptr) {
    if (!c->ut_valid) {
        int rc = project_current<real>(c, nullptr, c->cur);
        if (rc) return rc;
        c->ut_valid = true;
    }
    StageParams<real> p = make_params<real>(c);
    p.dt = dt;
    for (int n = 0; n < nsteps; ++n)
        for (int s = 0; s < 5; ++s) {
            p.ut_in = ut_buf<real>(c, c->cur);
            p.ut_out = ut_buf<real>(c, c->cur ^ 1);
            p.rkA = RK_A[s];
            p.rkB = RK_B[s];
            p.t = t0 + n * dt + RK_C[s] * dt;
            p.u_out = (n == nsteps - 1 && s == 4) ? u_out : nullptr;
            CUDA_TRY(c, d_stage(c, p, 1));
            c->cur ^= 1;
        }
    return ESDG_OK;
}

// Halo traces of a partition: the u~ records of one face of one element (Nfp
// node records of `wpr` 16-byte words each; the face's nodes are records
// Nq + f Nfp + k of the element, or fmap[f Nfp + k] for the DG-SBP method).
// Pack: entry i = 4 e + f of a local element e < K gathers into out; an entry
// out of range gives zeros.  Unpack: entry i = 4 g + f of ghost record g < G
// scatters from in; an entry out of range is skipped.
__device__ __forceinline__ int halo_node(const int* fmap, int Nq, int Nfp, int f, int k) {
    return fmap ? fmap[f * Nfp + k] : Nq + f * Nfp + k;
}

__global__ void k_halo_pack(const uint4* __restrict__ ut, const int* __restrict__ ent, int n, int nrec, int Nq,
                            int Nfp, int wpr, const int* __restrict__ fmap, int K, uint4* __restrict__ out) {
    const long long per = (long long)Nfp * wpr, total = (long long)n * per;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = int(t / per), r = int(t - (long long)i * per), k = r / wpr, w = r - k * wpr;
        const int x = ent[i], e = x >> 2, f = x & 3;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (x >= 0 && e < K && f < 3) v = ut[((long long)e * nrec + halo_node(fmap, Nq, Nfp, f, k)) * wpr + w];
        out[t] = v;
    }
}

__global__ void k_halo_unpack(uint4* __restrict__ ut, const int* __restrict__ ent, int n, int nrec, int Nq, int Nfp,
                              int wpr, const int* __restrict__ fmap, int Kpad, int G, const uint4* __restrict__ in) {
    const long long per = (long long)Nfp * wpr, total = (long long)n * per;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = int(t / per), r = int(t - (long long)i * per), k = r / wpr, w = r - k * wpr;
        const int x = ent[i], g = x >> 2, f = x & 3;
        if (x >= 0 && g < G && f < 3)
            ut[((long long)(Kpad + g) * nrec + halo_node(fmap, Nq, Nfp, f, k)) * wpr + w] = in[t];
    }
}

static bool valid(const esdg_ctx* c) { return c != nullptr; }

// The local mesh of block `part` of a px x py block partition of the quad grid
// (blocks of whole quads, so each quad's two triangles stay together): the
// owned elements in increasing global order, then the ghosts, i.e. elements of
// other blocks across a cut face, sorted by owning block and global element.
// Face neighbours become local indices; a ghost's u~ record is Kpad + g.
static bool restrict_mesh(const MeshData& F, const esdg_config& cfg, int px, int py, int part, MeshData& M,
                          std::vector<int>& owned, std::vector<int>& gg, std::vector<int>& gp, std::string& err) {
    const int nx = cfg.nx, ny = cfg.ny;
    // block b covers quads [b n / p, (b + 1) n / p) in each direction
    std::vector<int> bxq(nx, 0), byq(ny, 0);
    for (int b = 0; b < px; ++b)
        for (int i = int((long long)b * nx / px); i < int((long long)(b + 1) * nx / px); ++i) bxq[i] = b;
    for (int b = 0; b < py; ++b)
        for (int j = int((long long)b * ny / py); j < int((long long)(b + 1) * ny / py); ++j) byq[j] = b;
    auto block_of_quad = [&](int i, int j) { return byq[j] * px + bxq[i]; };
    std::vector<int> elem_part(size_t(F.K));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int b = block_of_quad(i, j);
            elem_part[2 * size_t(j * nx + i)] = elem_part[2 * size_t(j * nx + i) + 1] = b;
        }
    owned.clear();
    for (int e = 0; e < F.K; ++e)
        if (elem_part[e] == part) owned.push_back(e);
    const int K = int(owned.size());
    if (K == 0) { err = "empty partition block"; return false; }
    std::vector<int> local(size_t(F.K), -1);
    for (int k = 0; k < K; ++k) local[owned[k]] = k;
    std::vector<std::pair<int, int>> ghosts;  // (part, global element)
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < 3; ++f) {
            const int nb = F.nbr[3 * size_t(owned[k]) + f], en = nb >> 2;
            if ((nb & 3) != 3 && local[en] < 0) ghosts.push_back({elem_part[en], en});
        }
    std::sort(ghosts.begin(), ghosts.end());
    ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
    gg.clear();
    gp.clear();
    for (auto& g : ghosts) {
        gp.push_back(g.first);
        gg.push_back(g.second);
    }
    const int Kpad = (K + 7) / 8 * 8;
    std::vector<int> ghost_slot(size_t(F.K), -1);
    for (size_t g = 0; g < gg.size(); ++g) ghost_slot[gg[g]] = Kpad + int(g);
    auto take = [&](const std::vector<double>& v, std::vector<double>& out) {
        const size_t w = v.size() / size_t(F.K);
        out.resize(w * K);
        for (int k = 0; k < K; ++k) std::copy_n(v.begin() + w * owned[k], w, out.begin() + w * k);
    };
    M.K = K;
    take(F.xeq, M.xeq); take(F.yeq, M.yeq); take(F.xq, M.xq); take(F.yq, M.yq);
    take(F.xf, M.xf); take(F.yf, M.yf); take(F.geo, M.geo); take(F.Jq, M.Jq); take(F.minv, M.minv);
    M.nbr.resize(3 * size_t(K));
    for (int k = 0; k < K; ++k)
        for (int f = 0; f < 3; ++f) {
            const int nb = F.nbr[3 * size_t(owned[k]) + f], en = nb >> 2, fn = nb & 3;
            if (fn == 3) M.nbr[3 * k + f] = 4 * k + 3;
            else M.nbr[3 * k + f] = 4 * (local[en] >= 0 ? local[en] : ghost_slot[en]) + fn;
        }
    return true;
}

template <typename real>
static int stage_t(esdg_ctx* c, int s, double dt, double t0) {
    StageParams<real> p = make_params<real>(c);
    p.dt = dt;
    p.ut_in = ut_buf<real>(c, c->cur);
    p.ut_out = ut_buf<real>(c, c->cur ^ 1);
    p.rkA = RK_A[s];
    p.rkB = RK_B[s];
    p.t = t0 + RK_C[s] * dt;
    CUDA_TRY(c, d_stage(c, p, 1));
    c->cur ^= 1;
    return ESDG_OK;
}



extern "C" {

int esdg_build_operators(const esdg_config* cfg, esdg_ctx** out) {
    if (!cfg || !out) return fail(nullptr, ESDG_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->N < 1 || cfg->N > 5) return fail(nullptr, ESDG_EINVAL, "N must be in 1..5");
    if (cfg->precision != ESDG_FP32 && cfg->precision != ESDG_FP64)
        return fail(nullptr, ESDG_EINVAL, "precision must be ESDG_FP32 or ESDG_FP64");
    if (!(cfg->g > 0)) return fail(nullptr, ESDG_EINVAL, "g must be positive");
    if (cfg->forcing != ESDG_FORCING_NONE && cfg->forcing != ESDG_FORCING_MMS_SINE)
        return fail(nullptr, ESDG_EINVAL, "unknown forcing");
    if (cfg->volume_rule != ESDG_RULE_COLLAPSED && cfg->volume_rule != ESDG_RULE_SYMMETRIC)
        return fail(nullptr, ESDG_EINVAL, "unknown volume rule");
    if (cfg->boundary != ESDG_BOUNDARY_PERIODIC && cfg->boundary != ESDG_BOUNDARY_WALLS)
        return fail(nullptr, ESDG_EINVAL, "unknown boundary kind");
    if (cfg->mass != ESDG_MASS_EXACT && cfg->mass != ESDG_MASS_WEIGHT_ADJUSTED)
        return fail(nullptr, ESDG_EINVAL, "unknown inverse-mass kind");
    if (cfg->method != ESDG_METHOD_MODAL && cfg->method != ESDG_METHOD_SBP)
        return fail(nullptr, ESDG_EINVAL, "unknown method");
    if (cfg->method == ESDG_METHOD_SBP && (cfg->boundary != ESDG_BOUNDARY_PERIODIC || cfg->mass != ESDG_MASS_EXACT))
        return fail(nullptr, ESDG_EINVAL, "the DG-SBP scheme takes periodic boundaries and its diagonal mass matrix");
    if (cfg->dense != ESDG_DENSE_AUTO && cfg->dense != ESDG_DENSE_SIMT && cfg->dense != ESDG_DENSE_TENSOR)
        return fail(nullptr, ESDG_EINVAL, "unknown dense-operator kind");
    if (cfg->dense == ESDG_DENSE_TENSOR && !tc_available(*cfg))
        return fail(nullptr, ESDG_EINVAL,
                    "ESDG_DENSE_TENSOR needs the FP32 modal path with the stored inverse, Np <= 16 and Nq <= 16");
    esdg_ctx* c = new (std::nothrow) esdg_ctx();
    if (!c) return fail(nullptr, ESDG_ENOMEM, "out of host memory");
    c->cfg = *cfg;
    std::string err;
    if (!build_reference(cfg->N, cfg->method == ESDG_METHOD_SBP ? 2 : cfg->volume_rule, c->ref, err)) {
        delete c;
        return fail(nullptr, ESDG_EINVAL, err);
    }
    MeshSpec sp{cfg->nx, cfg->ny, cfg->x0, cfg->x1, cfg->y0, cfg->y1, cfg->warp_ax, cfg->warp_ay,
                cfg->boundary == ESDG_BOUNDARY_WALLS, cfg->mass == ESDG_MASS_WEIGHT_ADJUSTED};
    if (!build_mesh(c->ref, sp, c->mesh, err)) {
        delete c;
        return fail(nullptr, ESDG_EINVAL, err);
    }
    c->b_modal.assign(size_t(c->mesh.K) * c->ref.Np, 0.0);
    compute_layout(c);
    *out = c;
    return ESDG_OK;
}

int esdg_build_partition(const esdg_config* cfg, int px, int py, int part, esdg_ctx** out) {
    if (!cfg || !out) return fail(nullptr, ESDG_EINVAL, "null argument");
    *out = nullptr;
    if (px < 1 || py < 1 || part < 0 || part >= px * py)
        return fail(nullptr, ESDG_EINVAL, "partition: need px, py >= 1 and 0 <= part < px * py");
    if (px > cfg->nx || py > cfg->ny) return fail(nullptr, ESDG_EINVAL, "partition: more blocks than quads");
    esdg_ctx* full = nullptr;
    int rc = esdg_build_operators(cfg, &full);
    if (rc) return rc;
    esdg_ctx* c = new (std::nothrow) esdg_ctx();
    if (!c) {
        delete full;
        return fail(nullptr, ESDG_ENOMEM, "out of host memory");
    }
    c->cfg = full->cfg;
    c->ref = full->ref;
    c->px = px;
    c->py = py;
    c->part = part;
    c->K_global = full->mesh.K;
    std::string err;
    const bool ok = restrict_mesh(full->mesh, *cfg, px, py, part, c->mesh, c->owned_gid, c->ghost_gid, c->ghost_part,
                                  err);
    delete full;
    if (!ok) {
        delete c;
        return fail(nullptr, ESDG_EINVAL, "partition: " + err);
    }
    c->b_modal.assign(size_t(c->mesh.K) * c->ref.Np, 0.0);
    compute_layout(c);
    *out = c;
    return ESDG_OK;
}

int esdg_partition_info(const esdg_ctx* c, int* K_global, int* nghost, int* px, int* py, int* part,
                        size_t* trace_bytes) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (trace_bytes) *trace_bytes = real_size(c) * size_t(c->ref.Nfp) * 4;
    if (K_global) *K_global = c->K_global ? c->K_global : c->mesh.K;
    if (nghost) *nghost = int(c->ghost_gid.size());
    if (px) *px = c->px;
    if (py) *py = c->py;
    if (part) *part = c->part;
    return ESDG_OK;
}

int esdg_partition_maps(const esdg_ctx* cc, int* owned_gid, int* ghost_gid, int* ghost_part) {
    esdg_ctx* c = const_cast<esdg_ctx*>(cc);
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    const int K = c->mesh.K;
    if (owned_gid)
        for (int k = 0; k < K; ++k) owned_gid[k] = c->owned_gid.empty() ? k : c->owned_gid[k];
    for (size_t g = 0; g < c->ghost_gid.size(); ++g) {
        if (ghost_gid) ghost_gid[g] = c->ghost_gid[g];
        if (ghost_part) ghost_part[g] = c->ghost_part[g];
    }
    return ESDG_OK;
}

int esdg_get_neighbors(const esdg_ctx* c, int* nbr) {
    if (!valid(c) || !nbr) return fail(nullptr, ESDG_EINVAL, "null argument");
    std::copy(c->mesh.nbr.begin(), c->mesh.nbr.end(), nbr);
    return ESDG_OK;
}

int esdg_get_config(const esdg_ctx* c, esdg_config* out) {
    if (!valid(c) || !out) return fail(nullptr, ESDG_EINVAL, "null argument");
    *out = c->cfg;
    return ESDG_OK;
}

int esdg_sizes(const esdg_ctx* c, int* K, int* Np, int* Nq, int* Nfq, size_t* device_bytes) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (K) *K = c->mesh.K;
    if (Np) *Np = c->ref.Np;
    if (Nq) *Nq = c->ref.Nq;
    if (Nfq) *Nfq = c->ref.Nfq;
    if (device_bytes) *device_bytes = c->L.total;
    return ESDG_OK;
}

int esdg_attach_device(esdg_ctx* c, void* buffer, size_t bytes, void* stream) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (c->attached) return fail(c, ESDG_ESTATE, "device memory already attached");
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    if (buffer) {
        if (bytes < c->L.total) return fail(c, ESDG_ENOMEM, "device buffer smaller than esdg_sizes() requires");
        if (reinterpret_cast<uintptr_t>(buffer) % 256) return fail(c, ESDG_EINVAL, "device buffer not 256-byte aligned");
        c->dbuf = reinterpret_cast<unsigned char*>(buffer);
        c->owns_buffer = false;
    } else {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, c->L.total);
        if (e != cudaSuccess) return fail(c, ESDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        c->dbuf = reinterpret_cast<unsigned char*>(p);
        c->owns_buffer = true;
    }
    int dev = 0;
    CUDA_TRY(c, cudaGetDevice(&dev));
    CUDA_TRY(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(c, d_geometry(c));
    if (!c->prepared) {
        if (c->cfg.precision == ESDG_FP32)
            build_image<float>(c, nullptr, 0);
        else
            build_image<double>(c, nullptr, 0);
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->dbuf, c->image.data(), c->L.res, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->dbuf + c->L.res, 0, c->L.total - c->L.res, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    std::vector<unsigned char>().swap(c->image);
    c->prepared = false;
    c->ut_valid = false;
    c->attached = true;
    return ESDG_OK;
}

int esdg_prepare(esdg_ctx* c, const double* b_nodal, const double* q_volq, int mode) {
    if (!valid(c) || !q_volq) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (c->attached) return fail(c, ESDG_ESTATE, "esdg_prepare comes before esdg_attach_device");
    if (mode != ESDG_INIT_DEPTH && mode != ESDG_INIT_SURFACE) return fail(c, ESDG_EINVAL, "unknown init mode");
    if (b_nodal) modal_bathymetry(c, b_nodal);
    if (c->cfg.precision == ESDG_FP32)
        build_image<float>(c, q_volq, mode);
    else
        build_image<double>(c, q_volq, mode);
    c->prepared = true;
    return ESDG_OK;
}

int esdg_get_points(const esdg_ctx* c, int kind, double* x, double* y) {
    if (!valid(c) || !x || !y) return fail(nullptr, ESDG_EINVAL, "null argument");
    const MeshData& M = c->mesh;
    const std::vector<double>*px, *py;
    if (kind == ESDG_POINTS_NODAL) { px = &M.xeq; py = &M.yeq; }
    else if (kind == ESDG_POINTS_VOLQ) { px = &M.xq; py = &M.yq; }
    else if (kind == ESDG_POINTS_FACEQ) { px = &M.xf; py = &M.yf; }
    else return fail(const_cast<esdg_ctx*>(c), ESDG_EINVAL, "unknown point set");
    std::memcpy(x, px->data(), px->size() * 8);
    std::memcpy(y, py->data(), py->size() * 8);
    return ESDG_OK;
}

int esdg_set_bathymetry(esdg_ctx* c, const double* b_nodal) {
    if (!valid(c) || !b_nodal) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    modal_bathymetry(c, b_nodal);
    return upload_bathymetry(c);
}

int esdg_init_state(esdg_ctx* c, const double* b_nodal, const double* q_volq, int mode) {
    if (!valid(c) || !q_volq) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (mode != ESDG_INIT_DEPTH && mode != ESDG_INIT_SURFACE) return fail(c, ESDG_EINVAL, "unknown init mode");
    if (b_nodal) {
        int rc = esdg_set_bathymetry(c, b_nodal);
        if (rc) return rc;
    }
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    std::vector<double> u(3 * size_t(c->mesh.K) * c->ndof);
    project_host(c, q_volq, mode, u.data());
    return esdg_set_state(c, u.data(), 0);
}

int esdg_set_state(esdg_ctx* c, const double* u, int on_device) {
    if (!valid(c) || !u) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    size_t bytes = 8 * 3 * size_t(c->mesh.K) * c->ndof;
    CUDA_TRY(c, cudaMemcpyAsync(c->dbuf + c->L.u, u, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->dbuf + c->L.res, 0, bytes, c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->ut_valid = false;
    return ESDG_OK;
}

int esdg_copy_state(const esdg_ctx* cc, double* u, int on_device) {
    esdg_ctx* c = const_cast<esdg_ctx*>(cc);
    if (!valid(c) || !u) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    size_t bytes = 8 * 3 * size_t(c->mesh.K) * c->ndof;
    CUDA_TRY(c, cudaMemcpyAsync(u, c->dbuf + c->L.u, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return ESDG_OK;
}

int esdg_rhs(esdg_ctx* c, double t, const double* u_in, double* rhs_out) {
    if (c && !c->ghost_gid.empty())
        return fail(c, ESDG_ESTATE, "a partition with ghost elements advances by esdg_stage with a halo exchange");
    if (!valid(c) || !rhs_out) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    int rc = c->cfg.precision == ESDG_FP32 ? rhs_t<float>(c, t, u_in, rhs_out) : rhs_t<double>(c, t, u_in, rhs_out);
    if (rc) return rc;
    return check_status(c);
}

int esdg_step_async(esdg_ctx* c, int nsteps, double dt, double t0) {
    if (c && !c->ghost_gid.empty())
        return fail(c, ESDG_ESTATE, "a partition with ghost elements advances by esdg_stage with a halo exchange");
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (nsteps < 0) return fail(c, ESDG_EINVAL, "nsteps < 0");
    if (!(dt > 0)) esdg_dt(c, &dt);
    return c->cfg.precision == ESDG_FP32 ? step_t<float>(c, nsteps, dt, t0) : step_t<double>(c, nsteps, dt, t0);
}

// A host buffer the device can address directly (pinned or registered host
// memory, or managed memory): its device-side address, else nullptr.
static const void* device_view(const void* host) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost && a.type != cudaMemoryTypeManaged) return nullptr;
    return a.devicePointer;
}

int esdg_step_host(esdg_ctx* c, const double* u_host, int nsteps, double dt, double* t_inout, double* u_out_host) {
    if (c && !c->ghost_gid.empty())
        return fail(c, ESDG_ESTATE, "a partition with ghost elements advances by esdg_stage with a halo exchange");
    if (!valid(c) || !u_host || !u_out_host) return fail(nullptr, ESDG_EINVAL, "null argument");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (nsteps < 1) return fail(c, ESDG_EINVAL, "nsteps < 1");
    const double* din = static_cast<const double*>(device_view(u_host));
    double* dout = static_cast<double*>(const_cast<void*>(device_view(u_out_host)));
    if (!din || !dout)
        return fail(c, ESDG_EINVAL, "esdg_step_host: buffers must be host memory the device can address "
                                    "(cudaHostAlloc / cudaHostRegister or managed)");
    if (!(dt > 0)) esdg_dt(c, &dt);
    const double t0 = t_inout ? *t_inout : 0.0;
    const bool fp32 = c->cfg.precision == ESDG_FP32;
    // the projection kernel reads the state over the host link and stores it
    // as the RK state (residual zeroed); the last stage writes the result back
    c->cur = 0;
    int rc = fp32 ? project_current<float>(c, din, c->cur, true) : project_current<double>(c, din, c->cur, true);
    if (rc) return rc;
    c->ut_valid = true;
    rc = fp32 ? step_t<float>(c, nsteps, dt, t0, dout) : step_t<double>(c, nsteps, dt, t0, dout);
    if (rc) return rc;
    rc = check_status(c);
    if (rc) return rc;
    if (t_inout) *t_inout = t0 + nsteps * dt;
    return ESDG_OK;
}

int esdg_project(esdg_ctx* c) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    int rc = c->cfg.precision == ESDG_FP32 ? project_current<float>(c, nullptr, c->cur)
                                           : project_current<double>(c, nullptr, c->cur);
    if (rc) return rc;
    c->ut_valid = true;
    return ESDG_OK;
}

int esdg_stage(esdg_ctx* c, int stage, double dt, double t0) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (stage < 0 || stage > 4) return fail(c, ESDG_EINVAL, "stage must be 0..4");
    if (!(dt > 0)) return fail(c, ESDG_EINVAL, "dt must be positive");
    if (!c->ut_valid) return fail(c, ESDG_ESTATE, "call esdg_project (and exchange the halo) first");
    return c->cfg.precision == ESDG_FP32 ? stage_t<float>(c, stage, dt, t0) : stage_t<double>(c, stage, dt, t0);
}

static int halo_launch(esdg_ctx* c, bool pack, const int* ent, int n, const void* src, void* dst) {
    const int wpr = int(real_size(c) * 4 / 16);
    const int Nfp = c->ref.Nfp;
    const int* fmap = c->sbp ? reinterpret_cast<const int*>(c->dbuf + c->L.fmap) : nullptr;
    unsigned char* ut = c->dbuf + (c->cur == 0 ? c->L.ut0 : c->L.ut1);
    const long long total = (long long)n * Nfp * wpr;
    const int block = 256;
    const int grid = int(std::min<long long>((total + block - 1) / block, 4LL * (c->num_sms ? c->num_sms : 152)));
    if (pack)
        k_halo_pack<<<grid, block, 0, c->stream>>>(reinterpret_cast<const uint4*>(ut), ent, n, c->nrec, c->ref.Nq, Nfp,
                                                     wpr, fmap, c->mesh.K, static_cast<uint4*>(dst));
    else
        k_halo_unpack<<<grid, block, 0, c->stream>>>(reinterpret_cast<uint4*>(ut), ent, n, c->nrec, c->ref.Nq, Nfp,
                                                       wpr, fmap, c->Kpad, int(c->ghost_gid.size()),
                                                       static_cast<const uint4*>(src));
    CUDA_TRY(c, cudaGetLastError());
    return ESDG_OK;
}

int esdg_halo_pack(esdg_ctx* c, const int* faces_dev, int n, void* out_dev) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (n < 0 || (n > 0 && (!faces_dev || !out_dev))) return fail(c, ESDG_EINVAL, "halo pack: bad arguments");
    return n == 0 ? ESDG_OK : halo_launch(c, true, faces_dev, n, nullptr, out_dev);
}

int esdg_halo_unpack(esdg_ctx* c, const void* in_dev, const int* faces_dev, int n) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (n < 0 || (n > 0 && (!faces_dev || !in_dev))) return fail(c, ESDG_EINVAL, "halo unpack: bad arguments");
    return n == 0 ? ESDG_OK : halo_launch(c, false, faces_dev, n, in_dev, nullptr);
}

int esdg_check(esdg_ctx* c) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    return check_status(c);
}

int esdg_step(esdg_ctx* c, int nsteps, double dt, double* t_inout) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!(dt > 0)) esdg_dt(c, &dt);
    double t0 = t_inout ? *t_inout : 0.0;
    int rc = esdg_step_async(c, nsteps, dt, t0);
    if (rc) return rc;
    rc = check_status(c);
    if (rc) return rc;
    if (t_inout) *t_inout = t0 + nsteps * dt;
    return ESDG_OK;
}

int esdg_entropy(esdg_ctx* c, double t, double* entropy, double* mass, double* entropy_rate) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    const double* rhs = nullptr;
    if (entropy_rate) {
        double* r = reinterpret_cast<double*>(c->dbuf + c->L.rhs);
        int rc = esdg_rhs(c, t, nullptr, r);
        if (rc) return rc;
        rhs = r;
    }
    double* out = reinterpret_cast<double*>(c->dbuf + c->L.diag);
    if (c->sbp)
        CUDA_TRY(c, launch_entropy_nodal(c->mesh.K, c->ref.Nq, c->cfg.g, reinterpret_cast<const double*>(c->dbuf + c->L.u),
                                         rhs, reinterpret_cast<const double*>(c->dbuf + c->L.wJq64),
                                         reinterpret_cast<const double*>(c->dbuf + c->L.bq64),
                                         reinterpret_cast<double*>(c->dbuf + c->L.partial), c->entropy_parts, out,
                                         c->stream));
    else
        CUDA_TRY(c, d_entropy(kernel_nr(c->cfg), c->mesh.K, c->cfg.g, reinterpret_cast<const double*>(c->dbuf + c->L.u),
                              rhs, reinterpret_cast<const double*>(c->dbuf + c->L.vq64),
                              reinterpret_cast<const double*>(c->dbuf + c->L.wJq64),
                              reinterpret_cast<const double*>(c->dbuf + c->L.bq64),
                              reinterpret_cast<double*>(c->dbuf + c->L.partial), c->entropy_parts, out, c->stream));
    double h[3];
    CUDA_TRY(c, cudaMemcpyAsync(h, out, 24, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (entropy) *entropy = h[0];
    if (mass) *mass = h[1];
    if (entropy_rate) *entropy_rate = h[2];
    return ESDG_OK;
}

int esdg_l2_error(esdg_ctx* c, const double* exact_volq, double* err) {
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (!exact_volq || !err) return fail(c, ESDG_EINVAL, "exact_volq and err must not be NULL");
    cudaPointerAttributes attr;
    CUDA_TRY(c, cudaPointerGetAttributes(&attr, exact_volq));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(c, ESDG_EINVAL, "exact_volq must be device memory");
    double* out = reinterpret_cast<double*>(c->dbuf + c->L.diag);
    CUDA_TRY(c, launch_l2_error(c->mesh.K, c->ref.Nq, c->ndof, reinterpret_cast<const double*>(c->dbuf + c->L.u),
                                c->sbp ? nullptr : reinterpret_cast<const double*>(c->dbuf + c->L.vq64),
                                reinterpret_cast<const double*>(c->dbuf + c->L.wJq64), exact_volq,
                                reinterpret_cast<double*>(c->dbuf + c->L.partial), c->entropy_parts, out, c->stream));
    double h[3];
    CUDA_TRY(c, cudaMemcpyAsync(h, out, 24, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int f = 0; f < 3; ++f) err[f] = std::sqrt(h[f]);
    return ESDG_OK;
}

// ---- no-allocation variant of the entropy diagnostic --------------------------
// Scratch for the per-block partial sums (3 per block) and the 3 totals.
static __device__ __align__(256) double g_noalloc_scratch[ESDG_NOALLOC_MAX_PARTS * 3 + 4];

// The array's device address for the current device.  Host code cannot use the
// symbol itself (on the host it only names a stand-in), so every call looks the
// address up with the caller's device current: no cached pointer can outlive a
// device reset or a re-created primary context.  The lookup allocates nothing.
static int noalloc_scratch(esdg_ctx* c, double** out) {
    void* p = nullptr;
    CUDA_TRY(c, cudaGetSymbolAddress(&p, g_noalloc_scratch));
    *out = static_cast<double*>(p);
    return ESDG_OK;
}

// Whether K * Nq volume points fit the static scratch (host arithmetic only).
static bool noalloc_fits(long long points, long long* parts) {
    *parts = (points + ESDG_NOALLOC_POINTS_PER_PART - 1) / ESDG_NOALLOC_POINTS_PER_PART;
    return *parts <= ESDG_NOALLOC_MAX_PARTS;
}

int esdg_entropy_noalloc(const esdg_ctx* cc, const double* u_dev, double* entropy, double* mass) {
    esdg_ctx* c = const_cast<esdg_ctx*>(cc);
    if (!valid(c)) return fail(nullptr, ESDG_EINVAL, "null context");
    // the size limit is checked first, on the host, before any CUDA call
    const long long points = (long long)c->mesh.K * c->ref.Nq;
    long long parts = 0;
    if (!noalloc_fits(points, &parts))
        return fail(c, ESDG_EINVAL,
                    "esdg_entropy_noalloc: K * Nq = " + std::to_string(points) + " exceeds the static scratch limit of " +
                        std::to_string((long long)ESDG_NOALLOC_MAX_PARTS * ESDG_NOALLOC_POINTS_PER_PART) +
                        " quadrature points; use esdg_entropy");
    if (!c->attached) return fail(c, ESDG_ESTATE, "attach device memory first");
    if (u_dev) {
        // a host or stale pointer would fault inside the kernel: refuse it here
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, u_dev) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, ESDG_EINVAL, "esdg_entropy_noalloc: u_dev is not a CUDA pointer");
        }
        if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
            return fail(c, ESDG_EINVAL, "esdg_entropy_noalloc: u_dev must be device memory");
    }
    double* scratch = nullptr;
    int rc = noalloc_scratch(c, &scratch);
    if (rc) return rc;
    double* partial = scratch;
    double* out = scratch + ESDG_NOALLOC_MAX_PARTS * 3;
    const double* u = u_dev ? u_dev : reinterpret_cast<const double*>(c->dbuf + c->L.u);
    // every block writes its own partial and the finalize kernel writes all three
    // totals, so no part of the scratch has to start at zero
    if (c->sbp)
        CUDA_TRY(c, launch_entropy_nodal(c->mesh.K, c->ref.Nq, c->cfg.g, u, nullptr,
                                         reinterpret_cast<const double*>(c->dbuf + c->L.wJq64),
                                         reinterpret_cast<const double*>(c->dbuf + c->L.bq64), partial, (int)parts, out,
                                         c->stream));
    else
        CUDA_TRY(c, d_entropy(kernel_nr(c->cfg), c->mesh.K, c->cfg.g, u, nullptr,
                              reinterpret_cast<const double*>(c->dbuf + c->L.vq64),
                              reinterpret_cast<const double*>(c->dbuf + c->L.wJq64),
                              reinterpret_cast<const double*>(c->dbuf + c->L.bq64), partial, (int)parts, out,
                              c->stream));
    double h[3];
    CUDA_TRY(c, cudaMemcpyAsync(h, out, 24, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (entropy) *entropy = h[0];
    if (mass) *mass = h[1];
    return ESDG_OK;
}

// ---- ensembles ------------------------------------------------------------------
struct esdg_ensemble {
    std::vector<esdg_ctx*> members;
    std::vector<int> order;        // tile-table order of members
    EnsembleMember* dmem = nullptr;
    int total_batches = 0;
    int warps = 12;
    int nmax = 4;
    int4 ops_lo = make_int4(-1, -1, -1, -1);
    int ops_hi = -1, ops_end = 0, slab = 0;
    int rule = ESDG_RULE_COLLAPSED;  // shared by all members
    size_t smem = 0;
    cudaStream_t stream = nullptr;    // the members' stream (work and graph launches)
    cudaStream_t capture = nullptr;   // private stream the graph is captured on (the
                                      // legacy default stream cannot be captured)
    cudaGraphExec_t graph = nullptr;  // GRAPH_STEPS steps
    int graph_warps = 0;
    std::string err;
};
static const int GRAPH_STEPS = 10;  // even: a replay returns the u~ buffers to the same parity

static int efail(esdg_ensemble* e, int code, const std::string& m) {
    e->err = m;
    return code;
}
#define ECUDA_TRY(ens, call)                                                                       \
    do {                                                                                           \
        cudaError_t e__ = (call);                                                                  \
        if (e__ != cudaSuccess) return efail((ens), ESDG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

static int c2_w_end(int NR) {
    switch (NR) {
#define X(v) case v: return C2<v>::w_end;
        ESDG_FOR_EACH_NR(X)
#undef X
    }
    return 0;
}

// (Re)build the member table in the given order and the shared-memory plan.
static int ensemble_table(esdg_ensemble* e) {
    std::vector<EnsembleMember> h;
    int begin = 0, ops = 0, slab = 0, nmax = 1;
    int off[6] = {-1, -1, -1, -1, -1, -1};
    for (int idx : e->order) {
        esdg_ctx* c = e->members[idx];
        const int N = c->cfg.N, NR = kernel_nr(c->cfg);
        if (off[N] < 0) {
            off[N] = ops;
            ops += c2_ops_floats(NR);
        }
        slab = std::max(slab, c2_w_end(NR));
        nmax = std::max(nmax, N);
        EnsembleMember m;
        std::memset(&m, 0, sizeof(m));
        m.p = make_params<float>(c);
        esdg_dt(c, &m.p.dt);
        // the ensemble kernel applies the dense operators on the FP32 pipes
        m.ops2 = reinterpret_cast<const float*>(c->dbuf + (use_tc(c->cfg) ? c->L.ops2s : c->L.ops2));
        m.ut[0] = ut_buf<float>(c, 0);
        m.ut[1] = ut_buf<float>(c, 1);
        m.N = N;
        m.batch_begin = begin;
        m.nbatch = c->Kpad / 4;
        begin += m.nbatch;
        h.push_back(m);
    }
    e->total_batches = begin;
    e->ops_lo = make_int4(off[1], off[2], off[3], off[4]);
    e->ops_hi = off[5];
    e->ops_end = ops;
    e->slab = slab;
    e->nmax = nmax <= 4 ? 4 : 5;
    const int n = int(h.size());
    e->smem = 4 * (size_t(ops) + size_t(e->warps) * slab) + 4 * size_t((n + 1 + 3) & ~3) + (8 + sizeof(StageParams<float>)) * size_t(e->warps);
    ECUDA_TRY(e, cudaMemcpyAsync(e->dmem, h.data(), sizeof(EnsembleMember) * n, cudaMemcpyHostToDevice, e->stream));
    ECUDA_TRY(e, cudaStreamSynchronize(e->stream));
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return ESDG_OK;
}

static int ensemble_fits(esdg_ensemble* e, int warps) {
    const int n = int(e->members.size());
    size_t need = 4 * (size_t(e->ops_end) + size_t(warps) * e->slab) + 4 * size_t((n + 1 + 3) & ~3) + (8 + sizeof(StageParams<float>)) * size_t(warps);
    return need <= 232448;
}

static int ensemble_launch(esdg_ensemble* e, int which, int stage, cudaStream_t st) {
    const int sms = e->members[0]->num_sms;
    const int n = int(e->members.size());
    auto launch = e->rule == ESDG_RULE_SYMMETRIC ? launch_ensemble<1> : launch_ensemble<0>;
    ECUDA_TRY(e, launch(e->nmax, sms, e->warps * 32, e->smem, st, e->dmem, n, e->total_batches, which,
                                 RK_A[stage], RK_B[stage], e->ops_lo, e->ops_hi, e->ops_end, e->slab));
    return ESDG_OK;
}

// Make every member's u~ buffer 0 current for its state.
static int ensemble_prepare(esdg_ensemble* e) {
    for (esdg_ctx* c : e->members) {
        if (!c->ut_valid || c->cur != 0) {
            c->cur = 0;
            int rc = project_current<float>(c, nullptr, 0);
            if (rc) return efail(e, rc, c->err);
            c->ut_valid = true;
        }
    }
    return ESDG_OK;
}

static int ensemble_set_shape(esdg_ensemble* e, int warps) {
    e->warps = warps;
    const int n = int(e->members.size());
    e->smem = 4 * (size_t(e->ops_end) + size_t(warps) * e->slab) + 4 * size_t((n + 1 + 3) & ~3) + (8 + sizeof(StageParams<float>)) * size_t(warps);
    cudaError_t err = e->rule == ESDG_RULE_SYMMETRIC ? ensemble_smem_attr<1>(e->nmax, e->smem)
                                                     : ensemble_smem_attr<0>(e->nmax, e->smem);
    if (err != cudaSuccess) return efail(e, ESDG_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return ESDG_OK;
}

static int ensemble_steps_direct(esdg_ensemble* e, int nsteps, int* stage_counter, cudaStream_t st) {
    for (int k = 0; k < nsteps; ++k)
        for (int s = 0; s < 5; ++s) {
            int rc = ensemble_launch(e, (*stage_counter) & 1, s, st);
            if (rc) return rc;
            ++*stage_counter;
        }
    return ESDG_OK;
}

int esdg_ensemble_create(esdg_ctx* const* members, int n, esdg_ensemble** out) {
    if (!members || n < 1 || !out) return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: bad arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const esdg_ctx* c = members[i];
        if (!c || !c->attached) return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: member not attached");
        if (c->cfg.precision != ESDG_FP32) return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members must be FP32");
        if (c->cfg.forcing != ESDG_FORCING_NONE)
            return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members with a forcing term are not supported");
        if (c->stream != members[0]->stream)
            return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members must share one stream");
        if (c->cfg.volume_rule != members[0]->cfg.volume_rule)
            return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members must share one volume rule");
        if (weight_adjusted(c->cfg))
            return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members must use the stored inverse mass matrices");
        if (c->sbp) return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: members must use the modal scheme");
        if (!c->ghost_gid.empty())
            return fail(nullptr, ESDG_EINVAL, "esdg_ensemble_create: a block of a partition needs its halo exchange");
    }
    esdg_ensemble* e = new (std::nothrow) esdg_ensemble();
    if (!e) return fail(nullptr, ESDG_ENOMEM, "out of host memory");
    e->members.assign(members, members + n);
    e->stream = members[0]->stream;
    e->rule = members[0]->cfg.volume_rule;
    for (int i = 0; i < n; ++i) e->order.push_back(i);
    cudaError_t err = cudaMalloc(&e->dmem, sizeof(EnsembleMember) * n);
    if (err != cudaSuccess) {
        delete e;
        return fail(nullptr, ESDG_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(err));
    }
    err = cudaStreamCreateWithFlags(&e->capture, cudaStreamNonBlocking);
    if (err != cudaSuccess) {
        cudaFree(e->dmem);
        delete e;
        return fail(nullptr, ESDG_ECUDA, std::string("cudaStreamCreateWithFlags: ") + cudaGetErrorString(err));
    }
    int rc = ensemble_table(e);
    if (!rc) {
        int w = ensemble_max_warps(e->nmax);
        while (w > 1 && !ensemble_fits(e, w)) --w;
        rc = ensemble_set_shape(e, w);
    }
    if (rc) {
        std::string m = e->err;
        cudaFree(e->dmem);
        cudaStreamDestroy(e->capture);
        delete e;
        return fail(nullptr, rc, m);
    }
    *out = e;
    return ESDG_OK;
}

int esdg_ensemble_step_async(esdg_ensemble* e, int nsteps) {
    if (!e || nsteps < 0) return fail(nullptr, ESDG_EINVAL, "bad arguments");
    int rc = ensemble_prepare(e);
    if (rc) return rc;
    int stage = 0;
    const int reps = nsteps / GRAPH_STEPS;
    if (reps > 0) {
        if (!e->graph || e->graph_warps != e->warps) {
            if (e->graph) cudaGraphExecDestroy(e->graph);
            e->graph = nullptr;
            cudaGraph_t g = nullptr;
            ECUDA_TRY(e, cudaStreamBeginCapture(e->capture, cudaStreamCaptureModeThreadLocal));
            int st = 0;
            rc = ensemble_steps_direct(e, GRAPH_STEPS, &st, e->capture);
            cudaError_t ce = cudaStreamEndCapture(e->capture, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (ce != cudaSuccess) return efail(e, ESDG_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ce));
            ce = cudaGraphInstantiate(&e->graph, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return efail(e, ESDG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce));
            e->graph_warps = e->warps;
        }
        for (int r = 0; r < reps; ++r) ECUDA_TRY(e, cudaGraphLaunch(e->graph, e->stream));
    }
    rc = ensemble_steps_direct(e, nsteps - reps * GRAPH_STEPS, &stage, e->stream);
    if (rc) return rc;
    const int cur = (5 * nsteps) & 1;
    for (esdg_ctx* c : e->members) {
        c->cur = cur;
        c->ut_valid = true;
    }
    return ESDG_OK;
}

int esdg_ensemble_step(esdg_ensemble* e, int nsteps) {
    int rc = esdg_ensemble_step_async(e, nsteps);
    if (rc) return rc;
    ECUDA_TRY(e, cudaStreamSynchronize(e->stream));
    for (esdg_ctx* c : e->members) {
        rc = check_status(c);
        if (rc) return efail(e, rc, c->err);
    }
    return ESDG_OK;
}

int esdg_ensemble_autotune(esdg_ensemble* e, int* warps_out, int* order_out) {
    if (!e) return fail(nullptr, ESDG_EINVAL, "null ensemble");
    // keep each member's state in its own right-hand-side scratch; the RK
    // residual needs no saving (the first stage of a step does not read it)
    for (esdg_ctx* c : e->members)
        ECUDA_TRY(e, cudaMemcpyAsync(c->dbuf + c->L.rhs, c->dbuf + c->L.u, 8 * 3 * size_t(c->mesh.K) * c->ref.Np,
                                     cudaMemcpyDeviceToDevice, e->stream));
    std::vector<int> given = e->order, bydeg = e->order;
    std::stable_sort(bydeg.begin(), bydeg.end(),
                     [&](int a, int b) { return e->members[a]->cfg.N > e->members[b]->cfg.N; });
    float best = 1e30f;
    int best_w = e->warps, best_o = 0;
    cudaEvent_t t0, t1;
    ECUDA_TRY(e, cudaEventCreate(&t0));
    ECUDA_TRY(e, cudaEventCreate(&t1));
    int rc = ESDG_OK;
    for (int o = 0; o < 2 && !rc; ++o) {
        e->order = o == 0 ? given : bydeg;
        rc = ensemble_table(e);
        const int W = ensemble_max_warps(e->nmax);
        for (int w : {W - 4, W - 2, W}) {
            if (rc || !ensemble_fits(e, w)) continue;
            rc = ensemble_set_shape(e, w);
            if (!rc) rc = ensemble_prepare(e);
            int st = 0;
            if (!rc) rc = ensemble_steps_direct(e, 1, &st, e->stream);  // warm-up
            if (rc) break;
            cudaEventRecord(t0, e->stream);
            st = 0;
            rc = ensemble_steps_direct(e, 2, &st, e->stream);
            cudaEventRecord(t1, e->stream);
            cudaEventSynchronize(t1);
            float ms = 0;
            cudaEventElapsedTime(&ms, t0, t1);
            if (!rc && ms < best) {
                best = ms;
                best_w = w;
                best_o = o;
            }
            for (esdg_ctx* c : e->members) c->ut_valid = false;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (esdg_ctx* c : e->members) {
        ECUDA_TRY(e, cudaMemcpyAsync(c->dbuf + c->L.u, c->dbuf + c->L.rhs, 8 * 3 * size_t(c->mesh.K) * c->ref.Np,
                                     cudaMemcpyDeviceToDevice, e->stream));
        c->ut_valid = false;
    }
    if (rc) return rc;
    e->order = best_o == 0 ? given : bydeg;
    rc = ensemble_table(e);
    if (!rc) rc = ensemble_set_shape(e, best_w);
    if (rc) return rc;
    ECUDA_TRY(e, cudaStreamSynchronize(e->stream));
    for (esdg_ctx* c : e->members) {
        rc = check_status(c);
        if (rc) return efail(e, rc, c->err);
    }
    if (warps_out) *warps_out = best_w;
    if (order_out) *order_out = best_o;
    return ESDG_OK;
}

int esdg_ensemble_destroy(esdg_ensemble* e) {
    if (!e) return ESDG_OK;
    if (e->graph) cudaGraphExecDestroy(e->graph);
    if (e->dmem) cudaFree(e->dmem);
    if (e->capture) cudaStreamDestroy(e->capture);
    delete e;
    return ESDG_OK;
}

int esdg_dt(const esdg_ctx* c, double* dt) {
    if (!valid(c) || !dt) return fail(nullptr, ESDG_EINVAL, "null argument");
    const int N = c->cfg.N;
    double CN = 0.5 * (N + 1) * (N + 2);
    *dt = c->cfg.cfl * ((c->cfg.x1 - c->cfg.x0) / c->cfg.nx) / CN;
    return ESDG_OK;
}

int esdg_destroy(esdg_ctx* c) {
    if (!c) return ESDG_OK;
    if (c->owns_buffer && c->dbuf) cudaFree(c->dbuf);
    delete c;
    return ESDG_OK;
}

const char* esdg_last_error(const esdg_ctx* c) {
    return c ? c->err.c_str() : g_build_error.c_str();
}

const char* esdg_ensemble_error(const esdg_ensemble* e) {
    return e ? e->err.c_str() : g_build_error.c_str();
}

}  // extern "C"
