// DG-SBP kernels (Sec. 3 of Wu, Kubatko, Chan, arXiv 2005.02516) for sm_103a.
//
// The traditional entropy-stable DG-SBP scheme: nodal unknowns at the Nq
// points of an SBP rule (exact to 2N-1, the face Gauss-Legendre points among
// them), no entropy projection, the SBP operator Q_SBP = [I; I_f]^T Q_h [I; I_f]
// of Theorem 3.1 and the diagonal mass matrix W J.  Per element and stage,
// with the split form of Sec. 5.2 applied to Q_SBP (Q_SBP + Q_SBP^T =
// I_f^T B I_f, so 2 Q_SBP o F 1 = Qskew o F 1 + I_f^T B f(u_f)):
//   r_l = sum_m Qskew^{x,k}[l,m] f_S^x(u_l, u_m) + Qskew^{y,k}[l,m] f_S^y(u_l, u_m)
//         (+ the bathymetry source folded into the pressure as in esdg_kernels.cuh)
//       + [l = I_f(f)] w_f (nxJ f_S^x(u+, u_l) + nyJ f_S^y(u+, u_l)) - LF,
//   du_l/dt = -r_l / (w_l J_l) + forcing,
// then the LSRK45 stage.  Qskew^{i,k}[l,m] = sum_j Qskew_SBP^j[l,m] (G_ij[l] +
// G_ij[m]) / 2 with the metrics at the SBP nodes (a face node shares them with
// its volume node).  Neighbour values come from the previous stage's nodal
// record buffer (ut_in), so a stage never reads values it is updating.
//
// A warp per element (rows l = lane, lane + 32), operators in shared memory:
// the FP64 stages, and the preparation of nodal records from a state (MODE 2)
// in both precisions; the FP32 stages run on the batched k_sbp2
// (esdg_sbp2.cuh).
#pragma once

#include "esdg_kernels.cuh"

namespace esdg {

// Points of the SBP rule of degree N: 3(N+1) face Gauss-Legendre points plus
// the interior orbits.
constexpr int sbp_points(int N) { return N == 1 ? 6 : N == 2 ? 10 : N == 3 ? 18 : N == 4 ? 22 : 34; }

template <int N_>
struct SbpDims {
    static constexpr int N = N_;
    static constexpr int Np = (N + 1) * (N + 2) / 2;
    static constexpr int Nq = sbp_points(N);
    static constexpr int Nfp = N + 1;
    static constexpr int Nfq = 3 * (N + 1);
};

template <int N, typename real>
struct SbpSmem {
    typedef SbpDims<N> D;
    static constexpr int REC = 12;  // h hu hv u v H rx sx ry sy 2gh b
    static constexpr int ops_QsT = 0;                         // [Nq(m)][Nq(l)][2]
    static constexpr int ops_wf = ops_QsT + D::Nq * D::Nq * 2;
    static constexpr int ops_nrs = ops_wf + D::Nfq;
    static constexpr int ops_end = ((ops_nrs + 2 * D::Nfq) + 3) & ~3;
    static constexpr int w_rec = 0;                           // [Nq][REC]
    static constexpr int w_r = w_rec + D::Nq * REC;           // [3][Nq] du/dt
    // the pair loop in 32 equal pieces of the flattened Nq x Nq pair list:
    // each lane's piece spans at most PR rows, whose partial sums meet in
    // w_part ([32][PR][4]: three sums and the row)
    static constexpr int PL = (D::Nq * D::Nq + 31) / 32;      // pairs per lane
    static constexpr int PR = (PL + D::Nq - 2) / D::Nq + 1;   // rows a piece can touch
    static constexpr int w_part = w_r + 3 * D::Nq;
    static constexpr int w_end = ((w_part + 32 * PR * 4) + 3) & ~3;
    static constexpr size_t bytes(int warps) {
        return sizeof(real) * (size_t(ops_end) + size_t(warps) * w_end) + sizeof(int) * 2 * 64;
    }
};

// MODE 0: du/dt into rhs_out.  MODE 1: LSRK45 stage of (u, res), the new
// nodal records into ut_out.  MODE 2: nodal records of u_in into ut_out (and,
// with copy_in, u_in stored as the state with the residual zeroed).
template <int N, typename real, int MODE>
__global__ void __launch_bounds__(256) k_sbp(StageParams<real> p) {
    typedef SbpDims<N> D;
    typedef SbpSmem<N, real> S;
    typedef typename V2<real>::t real2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* ops = reinterpret_cast<real*>(smem_raw);
    const int wpb = blockDim.x >> 5;
    int* fmap = reinterpret_cast<int*>(ops + S::ops_end + wpb * S::w_end);  // [Nfq]
    int* frow = fmap + 64;                                                  // [Nq]: face node of row, or -1
    for (int i = threadIdx.x; i < D::Nq * D::Nq * 2; i += blockDim.x) ops[S::ops_QsT + i] = p.QsT[i];
    for (int i = threadIdx.x; i < D::Nfq; i += blockDim.x) {
        ops[S::ops_wf + i] = p.wf[i];
        ops[S::ops_nrs + 2 * i] = p.nrs[2 * i];
        ops[S::ops_nrs + 2 * i + 1] = p.nrs[2 * i + 1];
        fmap[i] = p.fmap[i];
    }
    for (int i = threadIdx.x; i < D::Nq; i += blockDim.x) frow[i] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < D::Nfq; i += blockDim.x) frow[fmap[i]] = i;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    real* ws = ops + S::ops_end + warp * S::w_end;
    real* rec = ws + S::w_rec;
    real* rr = ws + S::w_r;
    const real2* QsT = reinterpret_cast<const real2*>(ops + S::ops_QsT);
    const real g = p.g;
    const real eighth = real(0.125);
    for (int e = blockIdx.x * wpb + warp; e < p.K; e += gridDim.x * wpb) {
        if constexpr (MODE == 2) {
            int bad = 0;
            for (int i = lane; i < D::Nq; i += 32) {
                const size_t g0 = ((size_t)0 * p.K + e) * D::Nq + i;
                const size_t g1 = ((size_t)1 * p.K + e) * D::Nq + i;
                const size_t g2 = ((size_t)2 * p.K + e) * D::Nq + i;
                const double h = p.u_in[g0], hu = p.u_in[g1], hv = p.u_in[g2];
                if (p.copy_in) {
                    p.u[g0] = h;
                    p.u[g1] = hu;
                    p.u[g2] = hv;
                    p.res[g0] = p.res[g1] = p.res[g2] = 0.0;
                }
                if (!(h > 0.0)) bad |= STATUS_NONPOSITIVE;
                const double ih = 1.0 / h;
                const real hr = (real)h, ur = (real)(hu * ih), vr = (real)(hv * ih);
                real* o = p.ut_out + ((size_t)e * D::Nq + i) * 4;
                o[0] = hr;
                o[1] = ur;
                o[2] = vr;
                o[3] = hr + p.bh[(size_t)e * D::Nq + i];
            }
            if (bad) atomicOr(p.status, bad);
        } else {
        // ---- nodal records of the element ----------------------------------------
        for (int l = lane; l < D::Nq; l += 32) {
            const real* ut = p.ut_in + ((size_t)e * D::Nq + l) * 4;
            const real* gg = p.geo + ((size_t)e * D::Nq + l) * 4;
            const real h = ut[0], uu = ut[1], vv = ut[2], H = ut[3];
            const real b = p.bh[(size_t)e * D::Nq + l];
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
            r[11] = b;
        }
        __syncwarp();
        // ---- flux differencing over all node pairs --------------------------------
        // (u_l + u_m) T summed over m is u_l (sum of T) + sum of u_m T: the row
        // part is added once per row.  The Nq x Nq pairs, row-major, are cut
        // into 32 pieces of PL, one per lane (all lanes busy on the FP64 pipe,
        // which bounds the FP64 path); a piece's partial row sums go to w_part
        // when its row ends, and each row's owner adds up the pieces of its row.
        real* part = ws + S::w_part;
        {
            const int p0 = lane * S::PL;
            const int p1 = p0 + S::PL < D::Nq * D::Nq ? p0 + S::PL : D::Nq * D::Nq;
            int r = p0 < p1 ? p0 / D::Nq : 0, m = p0 < p1 ? p0 - r * D::Nq : 0, slot = 0;
            const real* rl = rec + r * S::REC;
            real hu_l = rl[1], hv_l = rl[2], gh2_l = rl[10];
            // c1p, c2p: sums of (Qx, Qy) H_m; the row's pressure terms are
            // 2 g h_l times them, added when the piece's row ends
            real c0 = 0, c1 = 0, c2 = 0, c1p = 0, c2p = 0;
            for (int k = 0; k < S::PR * 4; ++k) part[lane * S::PR * 4 + k] = real(-1);
            // the metric-averaged operator entries (Qskew^x, Qskew^y)[r][m] of
            // this lane's pairs, stored per element ([K][PL][32][2], formed on
            // the host: they depend on the geometry alone)
            const real* qe = p.qxy + ((size_t)e * S::PL * 32 + lane) * 2;
#pragma unroll 1
            for (int it = 0; it < S::PL; ++it) {
                const real2 Q = *reinterpret_cast<const real2*>(qe + 64 * it);
                if (p0 + it < p1) {
                    const real* rm = rec + m * S::REC;
                    const real Qx = Q.x, Qy = Q.y;
                    const real HU = hu_l + rm[1], HV = hv_l + rm[2];
                    const real T = Qx * HU + Qy * HV;
                    c0 += T;
                    c1 = fma(rm[3], T, c1);
                    c2 = fma(rm[4], T, c2);
                    c1p = fma(Qx, rm[5], c1p);
                    c2p = fma(Qy, rm[5], c2p);
                    if (++m == D::Nq || p0 + it + 1 == p1) {
                        // this row's piece ends: file its partial sums
                        real* o = part + (lane * S::PR + slot) * 4;
                        o[0] = c0;
                        o[1] = fma(gh2_l, c1p, c1);
                        o[2] = fma(gh2_l, c2p, c2);
                        o[3] = real(r);
                        ++slot;
                        c0 = c1 = c2 = c1p = c2p = 0;
                        if (m == D::Nq && r + 1 < D::Nq) {
                            m = 0;
                            ++r;
                            rl = rec + r * S::REC;
                            hu_l = rl[1]; hv_l = rl[2];
                            gh2_l = rl[10];
                        }
                    }
                }
            }
        }
        __syncwarp();
        for (int l = lane; l < D::Nq; l += 32) {
            const real* rl = rec + l * S::REC;
            const real h_l = rl[0], hu_l = rl[1], hv_l = rl[2], u_l = rl[3], v_l = rl[4];
            const real rx_l = rl[6], sx_l = rl[7], ry_l = rl[8], sy_l = rl[9];
            real a0 = 0, a1 = 0, a2 = 0;
            // the pieces of row l: lanes l Nq / PL .. ((l+1) Nq - 1) / PL, in lane order
            const int k0 = (l * D::Nq) / S::PL, k1 = ((l + 1) * D::Nq - 1) / S::PL;
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
            a1 += u_l * a0;
            a2 += v_l * a0;
            real r0 = real(2) * a0, r1 = a1, r2 = a2;
            const int f = frow[l];
            if (f >= 0) {
                const int face = f / D::Nfp, i = f - face * D::Nfp;
                const int nb = p.nbr[(size_t)e * 3 + face];
                const int en = nb >> 2, fn = nb & 3;
                const real nr = ops[S::ops_nrs + 2 * f], ns = ops[S::ops_nrs + 2 * f + 1];
                const real nxJ = real(8) * (rx_l * nr + sx_l * ns);
                const real nyJ = real(8) * (ry_l * nr + sy_l * ns);
                const real* up = p.ut_in + ((size_t)en * D::Nq + fmap[fn * D::Nfp + (D::Nfp - 1 - i)]) * 4;
                const real hP = up[0], uP = up[1], vP = up[2];
                const real huP = hP * uP, hvP = hP * vP;
                const real w = ops[S::ops_wf + f];
                const real b_l = rl[11];
                const real huA = real(0.5) * (hu_l + huP), hvA = real(0.5) * (hv_l + hvP);
                const real uA = real(0.5) * (u_l + uP), vA = real(0.5) * (v_l + vP);
                const real pw = real(0.5) * g * h_l * (hP + b_l);
                const real Fn0 = nxJ * huA + nyJ * hvA;
                r0 += w * Fn0;
                r1 += w * (uA * Fn0 + nxJ * pw);
                r2 += w * (vA * Fn0 + nyJ * pw);
                if (p.lf) {
                    // sJ max(|u.n| + sqrt(g h)) over both sides with the unit
                    // normal n = nJ / sJ folded in: |u.nJ| + sqrt(sJ^2 g h)
                    const real sJ2 = nxJ * nxJ + nyJ * nyJ;
                    const real lm = fabs(u_l * nxJ + v_l * nyJ) + r_sqrt(sJ2 * g * h_l);
                    const real lp = fabs(uP * nxJ + vP * nyJ) + r_sqrt(sJ2 * g * hP);
                    const real c = real(0.5) * w * (lm > lp ? lm : lp);
                    r0 -= c * (hP - h_l);
                    r1 -= c * (huP - hu_l);
                    r2 -= c * (hvP - hv_l);
                }
            }
            // du/dt = -r / (w J) + forcing (the forcing term W J f of the form, divided by W J)
            const real iwj = p.iwJ != nullptr ? p.iwJ[(size_t)e * D::Nq + l] : real(1) / p.wJq[(size_t)e * D::Nq + l];
            real d0 = -r0 * iwj, d1 = -r1 * iwj, d2 = -r2 * iwj;
            if (p.forcing) {
                const real x = p.xq[(size_t)e * D::Nq + l], y = p.yq[(size_t)e * D::Nq + l];
                real sth, cth, sx, cx, sy, cy;
                r_sincospi<real>(x + y - real(p.t), &sth, &cth);
                r_sincospi<real>(x, &sx, &cx);
                r_sincospi<real>(y, &sy, &cy);
                const real pi = real(3.14159265358979323846);
                const real h = real(2) + p.mms_amp * sth;
                const real c = p.mms_amp * pi * cth;
                const real bx = -p.mms_bamp * pi * sx * cy, by = -p.mms_bamp * pi * cx * sy;
                const real u0 = p.mms_u0, v0 = p.mms_v0;
                d0 += -c + u0 * c + v0 * c;
                d1 += -u0 * c + (u0 * u0 + g * h) * c + u0 * v0 * c + g * h * bx;
                d2 += -v0 * c + u0 * v0 * c + (v0 * v0 + g * h) * c + g * h * by;
            }
            rr[l] = d0;
            rr[D::Nq + l] = d1;
            rr[2 * D::Nq + l] = d2;
        }
        __syncwarp();
        // ---- output or LSRK45 stage (FP64) and the next stage's records ------------------
        int bad = 0;
        for (int l = lane; l < D::Nq; l += 32) {
            double un[3];
            for (int c = 0; c < 3; ++c) {
                const size_t gi = ((size_t)c * p.K + e) * D::Nq + l;
                const double d = (double)rr[c * D::Nq + l];
                if (MODE == 0) {
                    p.rhs_out[gi] = d;
                } else {
                    const double rs = p.rkA * p.res[gi] + p.dt * d;
                    p.res[gi] = rs;
                    un[c] = p.u[gi] + p.rkB * rs;
                    p.u[gi] = un[c];
                    if (p.u_out) p.u_out[gi] = un[c];
                }
            }
            if (MODE == 1) {
                const double h = un[0];
                if (!(h > 0.0)) bad |= STATUS_NONPOSITIVE;
                if (!isfinite(un[0]) || !isfinite(un[1]) || !isfinite(un[2])) bad |= STATUS_NONFINITE;
                const real hr = (real)h;
                const double ih = 1.0 / h;
                real* o = p.ut_out + ((size_t)e * D::Nq + l) * 4;
                o[0] = hr;
                o[1] = (real)(un[1] * ih);
                o[2] = (real)(un[2] * ih);
                o[3] = hr + rec[l * S::REC + 11];
            }
        }
        if (bad) atomicOr(p.status, bad);
        __syncwarp();
        }
    }
}



}  // namespace esdg
