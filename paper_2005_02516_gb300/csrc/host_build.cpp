// Host-side construction of the ESDG operators, mesh and geometry (FP64).
// Reference element: Sec. 2.1 (basis, quadrature, V_q, V_f, M, P_q, D^i),
// Sec. 2.2 (Q-hat^i = M D^i, B^i, Q^i, E, V_h), Sec. 2.3 (hybridized Q_h^i).
// Curved geometry: Sec. 2.7 (J, J-scaled G_ij, B^{i,k}, M_h^k); mesh warp: Sec. 4.
//
// Choices the paper leaves open (basis, rules, mesh) follow the conventions
// documented in esdg.h: orthonormal Dubiner basis, collapsed Gauss rule with
// (N+1)^2 points (exact to degree 2N+1), N+1 Gauss-Legendre points per face.

#include "host_build.hpp"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <cmath>
#include <map>
#include <utility>

namespace esdg {

// ---------------------------------------------------------------------------
// small dense linear algebra
// ---------------------------------------------------------------------------
Mat matmul(const Mat& A, const Mat& B) {
    Mat C(A.r, B.c);
    for (int i = 0; i < A.r; ++i)
        for (int k = 0; k < A.c; ++k) {
            double a = A(i, k);
            if (a == 0.0) continue;
            for (int j = 0; j < B.c; ++j) C(i, j) += a * B(k, j);
        }
    return C;
}

Mat transpose(const Mat& A) {
    Mat T(A.c, A.r);
    for (int i = 0; i < A.r; ++i)
        for (int j = 0; j < A.c; ++j) T(j, i) = A(i, j);
    return T;
}

bool invert(const Mat& A, Mat& Ainv) {
    const int n = A.r;
    Mat W = A;
    Ainv = Mat(n, n);
    for (int i = 0; i < n; ++i) Ainv(i, i) = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (std::fabs(W(i, col)) > std::fabs(W(piv, col))) piv = i;
        if (std::fabs(W(piv, col)) < 1e-300) return false;
        if (piv != col)
            for (int j = 0; j < n; ++j) {
                std::swap(W(piv, j), W(col, j));
                std::swap(Ainv(piv, j), Ainv(col, j));
            }
        double d = 1.0 / W(col, col);
        for (int j = 0; j < n; ++j) { W(col, j) *= d; Ainv(col, j) *= d; }
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            double f = W(i, col);
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) { W(i, j) -= f * W(col, j); Ainv(i, j) -= f * Ainv(col, j); }
        }
    }
    return true;
}

// Symmetric eigen-decomposition by cyclic Jacobi rotations (small n).
static void sym_eig(Mat A, std::vector<double>& evals, Mat& V) {
    const int n = A.r;
    V = Mat(n, n);
    for (int i = 0; i < n; ++i) V(i, i) = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += A(p, q) * A(p, q);
        if (off < 1e-40) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A(p, q);
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (A(q, q) - A(p, p)) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // A <- A R  (columns p, q)
                    double akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * akq;
                    A(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // A <- R^T A (rows p, q)
                    double apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * aqk;
                    A(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V(k, p), vkq = V(k, q);
                    V(k, p) = c * vkp - s * vkq;
                    V(k, q) = s * vkp + c * vkq;
                }
            }
    }
    evals.resize(n);
    for (int i = 0; i < n; ++i) evals[i] = A(i, i);
}

// ---------------------------------------------------------------------------
// Jacobi polynomials, orthonormal under (1-x)^alpha (1+x)^beta on [-1,1]
// ---------------------------------------------------------------------------
static double jacobi_mu0(double al, double be) {
    return std::pow(2.0, al + be + 1.0) * std::tgamma(al + 1.0) * std::tgamma(be + 1.0) /
           std::tgamma(al + be + 2.0);
}

// Three-term recurrence x p_n = a_{n+1} p_{n+1} + b_n p_n + a_n p_{n-1}.
static double rec_b(int n, double al, double be) {
    double s = 2.0 * n + al + be;
    if (n == 0) return (be - al) / (al + be + 2.0);
    return (be * be - al * al) / (s * (s + 2.0));
}
static double rec_a(int n, double al, double be) {  // n >= 1
    double s = 2.0 * n + al + be;
    double num = n * (n + al) * (n + be) * (n + al + be);
    double den = (s - 1.0) * (s + 1.0);
    if (n == 1) {  // n + al + be over s - 1 cancels exactly
        return 2.0 / s * std::sqrt((1.0 + al) * (1.0 + be) / (s + 1.0));
    }
    return 2.0 / s * std::sqrt(num / den);
}

static double jacobi_p(double x, double al, double be, int n) {
    double pm1 = 0.0, p = 1.0 / std::sqrt(jacobi_mu0(al, be));
    for (int k = 0; k < n; ++k) {
        double pn = ((x - rec_b(k, al, be)) * p - (k > 0 ? rec_a(k, al, be) * pm1 : 0.0)) / rec_a(k + 1, al, be);
        pm1 = p;
        p = pn;
    }
    return p;
}

// d/dx of the orthonormal p_n: sqrt(n (n+al+be+1)) p_{n-1}^{(al+1, be+1)}
static double jacobi_dp(double x, double al, double be, int n) {
    if (n == 0) return 0.0;
    return std::sqrt(n * (n + al + be + 1.0)) * jacobi_p(x, al + 1.0, be + 1.0, n - 1);
}

// Gauss-Jacobi rule with n points (Golub-Welsch).
static void gauss_jacobi(int n, double al, double be, std::vector<double>& x, std::vector<double>& w) {
    Mat T(n, n);
    for (int i = 0; i < n; ++i) {
        T(i, i) = rec_b(i, al, be);
        if (i + 1 < n) T(i, i + 1) = T(i + 1, i) = rec_a(i + 1, al, be);
    }
    std::vector<double> ev;
    Mat V;
    sym_eig(T, ev, V);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    double mu0 = jacobi_mu0(al, be);
    x.resize(n);
    w.resize(n);
    for (int i = 0; i < n; ++i) {
        int k = idx[i];
        double xi = ev[k];
        // one Newton correction on p_n for the last bits
        double p = jacobi_p(xi, al, be, n), dp = jacobi_dp(xi, al, be, n);
        if (dp != 0.0) xi -= p / dp;
        x[i] = xi;
        w[i] = mu0 * V(0, k) * V(0, k);
    }
}

// ---------------------------------------------------------------------------
// Dubiner basis (Sec. 2.1 leaves the basis open)
// ---------------------------------------------------------------------------
void dubiner(int N, const std::vector<double>& r, const std::vector<double>& s, Mat& V, Mat* Vr, Mat* Vs) {
    const int np = int(r.size());
    const int Np = (N + 1) * (N + 2) / 2;
    V = Mat(np, Np);
    if (Vr) *Vr = Mat(np, Np);
    if (Vs) *Vs = Mat(np, Np);
    const double rt2 = std::sqrt(2.0);
    for (int p = 0; p < np; ++p) {
        double b = s[p];
        double a = (std::fabs(1.0 - b) > 1e-14) ? 2.0 * (1.0 + r[p]) / (1.0 - b) - 1.0 : -1.0;
        int m = 0;
        for (int i = 0; i <= N; ++i)
            for (int j = 0; j <= N - i; ++j, ++m) {
                double fa = jacobi_p(a, 0.0, 0.0, i);
                double gb = jacobi_p(b, 2.0 * i + 1.0, 0.0, j);
                double omb_i = std::pow(1.0 - b, i);
                V(p, m) = rt2 * fa * gb * omb_i;
                if (!Vr) continue;
                // chain rule: d/dr = 2/(1-b) d/da, d/ds = (1+a)/(1-b) d/da + d/db
                double dfa = jacobi_dp(a, 0.0, 0.0, i);
                double dgb = jacobi_dp(b, 2.0 * i + 1.0, 0.0, j);
                double da_term = 0.0;   // (d phi/da) / (1-b) = sqrt2 fa' gb (1-b)^(i-1)
                if (i > 0) da_term = rt2 * dfa * gb * std::pow(1.0 - b, i - 1);
                double db = rt2 * fa * (dgb * omb_i - (i > 0 ? i * gb * std::pow(1.0 - b, i - 1) : 0.0));
                (*Vr)(p, m) = 2.0 * da_term;
                (*Vs)(p, m) = (1.0 + a) * da_term + db;
            }
    }
}

// ---------------------------------------------------------------------------
// Fully symmetric volume rules exact to degree 2N (positive weights, interior
// points).  Orbits of the triangle's symmetry group in barycentric coordinates:
// the centroid, (a, a, 1-2a) with its 3 permutations, (a, b, 1-a-b) with its
// 6.  Orbit counts (centroid, 3-point, 6-point) per degree 2N: 2: (0,1,0),
// 4: (0,2,0), 6: (0,2,1), 8: (1,3,1), 10: (1,2,3).  The parameters solve the
// moment equations sum_i w_i phi_k(x_i) = int phi_k over all basis functions
// of degree <= 2N, by Levenberg-Marquardt from seeded starting points; the
// solution is put in a canonical order (3-point orbits by a, 6-point orbits
// as a <= b <= c, by a).
// ---------------------------------------------------------------------------
namespace {
const int kSymStruct[6][3] = {{0, 0, 0}, {0, 1, 0}, {0, 2, 0}, {0, 2, 1}, {1, 3, 1}, {1, 2, 3}};

struct OrbitPoint {
    double lam[3];
    double w;
    int owner;          // index of the weight parameter
    int dpar[2];        // position parameters the point depends on (-1: none)
    double dlam[2][3];  // d lam / d parameter
};

std::vector<OrbitPoint> orbit_points(const std::vector<double>& th, const int st[3]) {
    std::vector<OrbitPoint> pts;
    int k = 0;
    if (st[0]) {
        OrbitPoint p{{1.0 / 3, 1.0 / 3, 1.0 / 3}, th[k], k, {-1, -1}, {{0, 0, 0}, {0, 0, 0}}};
        pts.push_back(p);
        k += 1;
    }
    for (int o = 0; o < st[1]; ++o) {
        const double a = th[k], c = 1 - 2 * a;
        const double L[3][3] = {{a, a, c}, {a, c, a}, {c, a, a}};
        const double D[3][3] = {{1, 1, -2}, {1, -2, 1}, {-2, 1, 1}};
        for (int q = 0; q < 3; ++q) {
            OrbitPoint p{{L[q][0], L[q][1], L[q][2]}, th[k + 1], k + 1, {k, -1}, {{D[q][0], D[q][1], D[q][2]}, {0, 0, 0}}};
            pts.push_back(p);
        }
        k += 2;
    }
    for (int o = 0; o < st[2]; ++o) {
        const double v[3] = {th[k], th[k + 1], 1 - th[k] - th[k + 1]};
        const double da[3] = {1, 0, -1}, db[3] = {0, 1, -1};
        const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
        for (int q = 0; q < 6; ++q) {
            OrbitPoint p;
            for (int i = 0; i < 3; ++i) {
                p.lam[i] = v[perm[q][i]];
                p.dlam[0][i] = da[perm[q][i]];
                p.dlam[1][i] = db[perm[q][i]];
            }
            p.w = th[k + 2];
            p.owner = k + 2;
            p.dpar[0] = k;
            p.dpar[1] = k + 1;
            pts.push_back(p);
        }
        k += 3;
    }
    return pts;
}

// r = -l1 + l2 - l3, s = -l1 - l2 + l3 (vertices (-1,-1), (1,-1), (-1,1))
inline double to_r(const double* l) { return -l[0] + l[1] - l[2]; }
inline double to_s(const double* l) { return -l[0] - l[1] + l[2]; }

uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double uniform(uint64_t& x, double lo, double hi) { return lo + (hi - lo) * (splitmix(x) >> 11) * (1.0 / 9007199254740992.0); }

bool sym_try(int N, uint64_t seed, std::vector<double>& th) {
    const int d = 2 * N;
    const int* st = kSymStruct[N];
    const int n = st[0] + 2 * st[1] + 3 * st[2];
    const int nm = (d + 1) * (d + 2) / 2;
    uint64_t x = seed * 7919 + 17;
    th.clear();
    if (st[0]) th.push_back(uniform(x, 0.05, 0.3));
    for (int o = 0; o < st[1]; ++o) { th.push_back(uniform(x, 0.02, 0.48)); th.push_back(uniform(x, 0.02, 0.3)); }
    for (int o = 0; o < st[2]; ++o) {
        th.push_back(uniform(x, 0.01, 0.45));
        th.push_back(uniform(x, 0.01, 0.45));
        th.push_back(uniform(x, 0.02, 0.2));
    }
    auto eval = [&](const std::vector<double>& t, std::vector<double>& R, Mat& J) {
        std::vector<OrbitPoint> pts = orbit_points(t, st);
        std::vector<double> r(pts.size()), s(pts.size());
        for (size_t i = 0; i < pts.size(); ++i) { r[i] = to_r(pts[i].lam); s[i] = to_s(pts[i].lam); }
        Mat V, Vr, Vs;
        dubiner(d, r, s, V, &Vr, &Vs);
        R.assign(nm, 0.0);
        J = Mat(nm, n);
        for (size_t i = 0; i < pts.size(); ++i)
            for (int m = 0; m < nm; ++m) {
                R[m] += pts[i].w * V(int(i), m);
                J(m, pts[i].owner) += V(int(i), m);
                for (int q = 0; q < 2; ++q) {
                    if (pts[i].dpar[q] < 0) continue;
                    const double dr = to_r(pts[i].dlam[q]), ds = to_s(pts[i].dlam[q]);
                    J(m, pts[i].dpar[q]) += pts[i].w * (Vr(int(i), m) * dr + Vs(int(i), m) * ds);
                }
            }
        R[0] -= std::sqrt(2.0);  // int over the triangle (area 2) of the constant mode 1/sqrt(2)
    };
    auto norm = [](const std::vector<double>& v) { double a = 0; for (double y : v) a += y * y; return std::sqrt(a); };
    std::vector<double> R, R2;
    Mat J, J2;
    eval(th, R, J);
    double mu = 1e-3;
    for (int it = 0; it < 200 && norm(R) > 1e-15; ++it) {
        Mat A(n, n), Ai;
        std::vector<double> g(n, 0.0);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                double sum = 0;
                for (int m = 0; m < nm; ++m) sum += J(m, i) * J(m, j);
                A(i, j) = sum + (i == j ? mu : 0.0);
            }
            for (int m = 0; m < nm; ++m) g[i] -= J(m, i) * R[m];
        }
        if (!invert(A, Ai)) { mu *= 10; continue; }
        std::vector<double> t2(th);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) t2[i] += Ai(i, j) * g[j];
        eval(t2, R2, J2);
        if (norm(R2) < norm(R)) {
            th = t2; R = R2; J = J2;
            mu = std::max(mu / 3, 1e-15);
        } else {
            mu *= 10;
            if (mu > 1e10) break;
        }
    }
    if (norm(R) > 1e-13) return false;
    for (const OrbitPoint& p : orbit_points(th, st)) {
        const double r = to_r(p.lam), s = to_s(p.lam);
        if (!(p.w > 0) || !(r > -1) || !(s > -1) || !(r + s < 0)) return false;
    }
    return true;
}
}  // namespace

// Canonical order of the orbit parameters: S21 by a; each S111 as a <= b <= c, by a.
static std::vector<double> sym_canonical(const std::vector<double>& th, const int* st) {
    std::vector<double> c;
    int k = 0;
    if (st[0]) c.push_back(th[k++]);
    std::vector<std::pair<double, double>> s21;
    for (int o = 0; o < st[1]; ++o, k += 2) s21.push_back({th[k], th[k + 1]});
    std::sort(s21.begin(), s21.end());
    std::vector<std::vector<double>> s111;
    for (int o = 0; o < st[2]; ++o, k += 3) {
        double v[3] = {th[k], th[k + 1], 1 - th[k] - th[k + 1]};
        std::sort(v, v + 3);
        s111.push_back({v[0], v[1], th[k + 2]});
    }
    std::sort(s111.begin(), s111.end());
    for (auto& p : s21) { c.push_back(p.first); c.push_back(p.second); }
    for (auto& q : s111) for (double v : q) c.push_back(v);
    return c;
}

// The moment equations can have several positive interior solutions (degree
// 10 has at least four): of those found from kSymRestarts seeded starts, take
// the one whose smallest weight is largest.
static const int kSymRestarts = 64;

bool symmetric_rule(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w, std::string& err) {
    if (N < 1 || N > 5) { err = "symmetric rules exist here for N = 1..5"; return false; }
    // one search per degree and process; later builds reuse it
    static std::mutex mu;
    static std::vector<double> cache[6];
    std::lock_guard<std::mutex> lock(mu);
    const int* st = kSymStruct[N];
    std::vector<double>& best = cache[N];
    if (best.empty()) {
        // restarts run on host threads; the choice below goes in seed order
        std::vector<std::vector<double>> found(kSymRestarts);
        std::vector<char> ok(kSymRestarts, 0);
        const int nt = std::max(1, std::min<int>(16, int(std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t]() {
                for (int seed = t; seed < kSymRestarts; seed += nt) ok[seed] = sym_try(N, uint64_t(seed), found[seed]);
            });
        for (auto& th : pool) th.join();
        double best_min = -1.0;
        for (int seed = 0; seed < kSymRestarts; ++seed) {
            if (!ok[seed]) continue;
            double wmin = 1e300;
            for (const OrbitPoint& p : orbit_points(found[seed], st)) wmin = std::min(wmin, p.w);
            if (wmin > best_min + 1e-12) {
                best_min = wmin;
                best = sym_canonical(found[seed], st);
            }
        }
        if (best.empty()) { err = "no symmetric volume rule found"; return false; }
    }
    r.clear(); s.clear(); w.clear();
    for (const OrbitPoint& p : orbit_points(best, st)) {
        r.push_back(to_r(p.lam));
        s.push_back(to_s(p.lam));
        w.push_back(p.w);
    }
    return true;
}

// ---------------------------------------------------------------------------
// SBP volume rules (Sec. 3.1): positive weights, exact to degree 2N-1, and the
// N+1 Gauss-Legendre points of every face among the nodes.  Fully symmetric:
// edge orbits at the fixed Gauss-Legendre points (the three edge midpoints
// when N+1 is odd, then one 6-point orbit per point t > 0, by increasing t)
// with free weights, then interior orbits (centroid, 3-point, 6-point counts
// per N: 1: none, 2: (1,0,0), 3: (0,0,1), 4: (1,2,0), 5: (1,1,2)), so that the
// symmetric moment equations of degree 2N-1 form a square system.  Solved by
// Levenberg-Marquardt from seeded starts like the rules above; each of these
// structures has a single positive interior solution.
// ---------------------------------------------------------------------------
namespace {
const int kSbpStruct[6][3] = {{0, 0, 0}, {0, 0, 0}, {1, 0, 0}, {0, 0, 1}, {1, 2, 0}, {1, 1, 2}};

// Edge orbit points (barycentric) of degree N with their weight index.
int sbp_edge_points(int N, const std::vector<double>& th, std::vector<OrbitPoint>& pts) {
    std::vector<double> t, w;
    gauss_jacobi(N + 1, 0.0, 0.0, t, w);
    int k = 0;
    if ((N + 1) % 2 == 1) {
        const double L[3][3] = {{0.5, 0.5, 0.0}, {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}};
        for (int q = 0; q < 3; ++q)
            pts.push_back(OrbitPoint{{L[q][0], L[q][1], L[q][2]}, th[k], k, {-1, -1}, {{0, 0, 0}, {0, 0, 0}}});
        k += 1;
    }
    std::vector<double> tp;
    for (double x : t)
        if (x > 1e-12) tp.push_back(x);
    std::sort(tp.begin(), tp.end());
    for (double x : tp) {
        const double a = 0.5 * (1.0 - x), b = 1.0 - a;
        const double L[6][3] = {{a, b, 0}, {b, a, 0}, {0, a, b}, {0, b, a}, {a, 0, b}, {b, 0, a}};
        for (int q = 0; q < 6; ++q)
            pts.push_back(OrbitPoint{{L[q][0], L[q][1], L[q][2]}, th[k], k, {-1, -1}, {{0, 0, 0}, {0, 0, 0}}});
        k += 1;
    }
    return k;
}

int sbp_edge_params(int N) { return (N + 1) % 2 + (N + 1) / 2; }

// All points of an SBP rule: edge orbits, then the interior orbits whose
// parameters follow the edge weights in th.
std::vector<OrbitPoint> sbp_points(int N, const std::vector<double>& th) {
    std::vector<OrbitPoint> pts;
    const int ne = sbp_edge_points(N, th, pts);
    const std::vector<double> ti(th.begin() + ne, th.end());
    for (OrbitPoint p : orbit_points(ti, kSbpStruct[N])) {
        p.owner += ne;
        for (int q = 0; q < 2; ++q)
            if (p.dpar[q] >= 0) p.dpar[q] += ne;
        pts.push_back(p);
    }
    return pts;
}

bool sbp_try(int N, uint64_t seed, std::vector<double>& th) {
    const int d = 2 * N - 1;
    const int* st = kSbpStruct[N];
    const int ne = sbp_edge_params(N);
    const int n = ne + st[0] + 2 * st[1] + 3 * st[2];
    const int nm = (d + 1) * (d + 2) / 2;
    uint64_t x = seed * 104729 + 31;
    th.clear();
    for (int i = 0; i < ne; ++i) th.push_back(uniform(x, 0.01, 0.2));
    if (st[0]) th.push_back(uniform(x, 0.05, 0.3));
    for (int o = 0; o < st[1]; ++o) { th.push_back(uniform(x, 0.02, 0.48)); th.push_back(uniform(x, 0.02, 0.3)); }
    for (int o = 0; o < st[2]; ++o) {
        th.push_back(uniform(x, 0.01, 0.45));
        th.push_back(uniform(x, 0.01, 0.45));
        th.push_back(uniform(x, 0.02, 0.2));
    }
    auto eval = [&](const std::vector<double>& t, std::vector<double>& R, Mat& J) {
        std::vector<OrbitPoint> pts = sbp_points(N, t);
        std::vector<double> r(pts.size()), s(pts.size());
        for (size_t i = 0; i < pts.size(); ++i) { r[i] = to_r(pts[i].lam); s[i] = to_s(pts[i].lam); }
        Mat V, Vr, Vs;
        dubiner(d, r, s, V, &Vr, &Vs);
        R.assign(nm, 0.0);
        J = Mat(nm, n);
        for (size_t i = 0; i < pts.size(); ++i)
            for (int m = 0; m < nm; ++m) {
                R[m] += pts[i].w * V(int(i), m);
                J(m, pts[i].owner) += V(int(i), m);
                for (int q = 0; q < 2; ++q) {
                    if (pts[i].dpar[q] < 0) continue;
                    const double dr = to_r(pts[i].dlam[q]), ds = to_s(pts[i].dlam[q]);
                    J(m, pts[i].dpar[q]) += pts[i].w * (Vr(int(i), m) * dr + Vs(int(i), m) * ds);
                }
            }
        R[0] -= std::sqrt(2.0);
    };
    auto norm = [](const std::vector<double>& v) { double a = 0; for (double y : v) a += y * y; return std::sqrt(a); };
    std::vector<double> R, R2;
    Mat J, J2;
    eval(th, R, J);
    double mu = 1e-3;
    for (int it = 0; it < 300 && norm(R) > 1e-15; ++it) {
        Mat A(n, n), Ai;
        std::vector<double> g(n, 0.0);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) {
                double sum = 0;
                for (int m = 0; m < nm; ++m) sum += J(m, i) * J(m, j);
                A(i, j) = sum + (i == j ? mu : 0.0);
            }
            for (int m = 0; m < nm; ++m) g[i] -= J(m, i) * R[m];
        }
        if (!invert(A, Ai)) { mu *= 10; if (mu > 1e10) break; continue; }
        std::vector<double> t2(th);
        bool finite = true;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) t2[i] += Ai(i, j) * g[j];
            finite = finite && std::isfinite(t2[i]);
        }
        if (!finite) return false;
        eval(t2, R2, J2);
        if (norm(R2) < norm(R)) {
            th = t2; R = R2; J = J2;
            mu = std::max(mu / 3, 1e-15);
        } else {
            mu *= 10;
            if (mu > 1e10) break;
        }
    }
    if (!(norm(R) < 1e-13)) return false;
    const std::vector<OrbitPoint> pts = sbp_points(N, th);
    const int nedge = 3 * ((N + 1) % 2) + 6 * ((N + 1) / 2);
    for (size_t i = 0; i < pts.size(); ++i) {
        if (!(pts[i].w > 0)) return false;
        if (int(i) < nedge) continue;
        const double r = to_r(pts[i].lam), s = to_s(pts[i].lam);
        if (!(r > -1 + 1e-9) || !(s > -1 + 1e-9) || !(r + s < -1e-9)) return false;
    }
    return true;
}
}  // namespace

bool sbp_rule(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w, std::string& err) {
    if (N < 1 || N > 5) { err = "SBP rules exist here for N = 1..5"; return false; }
    static std::mutex mu;
    static std::vector<double> cache[6];
    std::lock_guard<std::mutex> lock(mu);
    const int* st = kSbpStruct[N];
    const int ne = sbp_edge_params(N);
    std::vector<double>& best = cache[N];
    if (best.empty()) {
        std::vector<std::vector<double>> found(kSymRestarts);
        std::vector<char> ok(kSymRestarts, 0);
        const int nt = std::max(1, std::min<int>(16, int(std::thread::hardware_concurrency())));
        std::vector<std::thread> pool;
        for (int t = 0; t < nt; ++t)
            pool.emplace_back([&, t]() {
                for (int seed = t; seed < kSymRestarts; seed += nt) ok[seed] = sbp_try(N, uint64_t(seed), found[seed]);
            });
        for (auto& th : pool) th.join();
        double best_min = -1.0;
        for (int seed = 0; seed < kSymRestarts; ++seed) {
            if (!ok[seed]) continue;
            double wmin = 1e300;
            for (const OrbitPoint& p : sbp_points(N, found[seed])) wmin = std::min(wmin, p.w);
            if (wmin > best_min + 1e-12) {
                best_min = wmin;
                const std::vector<double> ti(found[seed].begin() + ne, found[seed].end());
                best.assign(found[seed].begin(), found[seed].begin() + ne);
                if (!ti.empty()) {
                    const std::vector<double> c = sym_canonical(ti, st);
                    best.insert(best.end(), c.begin(), c.end());
                }
            }
        }
        if (best.empty()) { err = "no SBP volume rule found"; return false; }
    }
    r.clear(); s.clear(); w.clear();
    for (const OrbitPoint& p : sbp_points(N, best)) {
        r.push_back(to_r(p.lam));
        s.push_back(to_s(p.lam));
        w.push_back(p.w);
    }
    return true;
}

// ---------------------------------------------------------------------------
// Reference element
// ---------------------------------------------------------------------------
bool build_reference(int N, int rule, RefOps& R, std::string& err) {
    if (N < 1 || N > 5) { err = "N must be in 1..5"; return false; }
    R.N = N;
    R.Np = (N + 1) * (N + 2) / 2;
    R.Nfp = N + 1;
    R.Nfq = 3 * R.Nfp;
    // volume: collapsed Gauss-Legendre (a) x Gauss-Jacobi(1,0) (b), (N+1)^2
    // points, or the fully symmetric rule exact to degree 2N
    std::vector<double> xa, wa, xb, wb;
    gauss_jacobi(N + 1, 0.0, 0.0, xa, wa);
    gauss_jacobi(N + 1, 1.0, 0.0, xb, wb);
    R.rq.clear(); R.sq.clear(); R.wq.clear();
    if (rule == 0) {
        for (int ia = 0; ia <= N; ++ia)
            for (int ib = 0; ib <= N; ++ib) {
                R.rq.push_back(0.5 * (1.0 + xa[ia]) * (1.0 - xb[ib]) - 1.0);
                R.sq.push_back(xb[ib]);
                R.wq.push_back(0.5 * wa[ia] * wb[ib]);
            }
    } else if (rule == 1) {
        if (!symmetric_rule(N, R.rq, R.sq, R.wq, err)) return false;
    } else if (!sbp_rule(N, R.rq, R.sq, R.wq, err)) {
        return false;
    }
    R.Nq = int(R.rq.size());
    R.Nh = R.Nq + R.Nfq;
    // faces: parameter t runs v1->v2, v2->v3, v3->v1 (counter-clockwise)
    R.rf.clear(); R.sf.clear(); R.wf.clear(); R.nr.clear(); R.ns.clear();
    for (int f = 0; f < 3; ++f)
        for (int i = 0; i <= N; ++i) {
            double t = xa[i];
            double rr = (f == 0) ? t : (f == 1 ? -t : -1.0);
            double ss = (f == 0) ? -1.0 : (f == 1 ? t : -t);
            R.rf.push_back(rr);
            R.sf.push_back(ss);
            R.wf.push_back(wa[i]);
            R.nr.push_back(f == 0 ? 0.0 : (f == 1 ? 1.0 : -1.0));
            R.ns.push_back(f == 0 ? -1.0 : (f == 1 ? 1.0 : 0.0));
        }
    // SBP rule: the volume node at each face node (the selection I_f, Sec. 3.2)
    R.fmap.clear();
    if (rule == 2)
        for (int f = 0; f < R.Nfq; ++f) {
            int best = -1;
            for (int q = 0; q < R.Nq; ++q)
                if (std::hypot(R.rq[q] - R.rf[f], R.sq[q] - R.sf[f]) < 1e-12) best = q;
            if (best < 0) { err = "a face node is not a node of the SBP rule"; return false; }
            R.fmap.push_back(best);
        }
    dubiner(N, R.rq, R.sq, R.Vq, &R.Vqr, &R.Vqs);
    dubiner(N, R.rf, R.sf, R.Vf, &R.Vfr, &R.Vfs);
    // M = Vq^T W Vq, Pq = M^{-1} Vq^T W
    Mat VqTW = transpose(R.Vq);
    for (int n = 0; n < R.Np; ++n)
        for (int q = 0; q < R.Nq; ++q) VqTW(n, q) *= R.wq[q];
    Mat M = matmul(VqTW, R.Vq), Minv;
    if (!invert(M, Minv)) { err = "singular reference mass matrix"; return false; }
    R.Pq = matmul(Minv, VqTW);
    // D^i = Pq Vq^i (derivatives of degree-N polynomials are degree N-1), Q-hat = M D
    Mat Qrh = matmul(M, matmul(R.Pq, R.Vqr));
    Mat Qsh = matmul(M, matmul(R.Pq, R.Vqs));
    // nodal Q^i = Pq^T Q-hat^i Pq, E = Vf Pq
    Mat PqT = transpose(R.Pq);
    Mat Qr = matmul(PqT, matmul(Qrh, R.Pq));
    Mat Qs = matmul(PqT, matmul(Qsh, R.Pq));
    Mat E = matmul(R.Vf, R.Pq);
    // skew hybridized operators Q_h - Q_h^T = [[Q - Q^T, E^T B], [-B E, 0]]
    auto skew = [&](const Mat& Q, const std::vector<double>& nh) {
        Mat S(R.Nh, R.Nh);
        for (int i = 0; i < R.Nq; ++i)
            for (int j = 0; j < R.Nq; ++j) S(i, j) = Q(i, j) - Q(j, i);
        for (int f = 0; f < R.Nfq; ++f) {
            double bf = R.wf[f] * nh[f];
            for (int j = 0; j < R.Nq; ++j) {
                S(j, R.Nq + f) = E(f, j) * bf;
                S(R.Nq + f, j) = -bf * E(f, j);
            }
        }
        return S;
    };
    R.Qsr = skew(Qr, R.nr);
    R.Qss = skew(Qs, R.ns);
    R.Vh = Mat(R.Nh, R.Np);
    for (int i = 0; i < R.Nq; ++i)
        for (int n = 0; n < R.Np; ++n) R.Vh(i, n) = R.Vq(i, n);
    for (int f = 0; f < R.Nfq; ++f)
        for (int n = 0; n < R.Np; ++n) R.Vh(R.Nq + f, n) = R.Vf(f, n);
    // equispaced nodes (s-major) and the inverse Vandermonde
    R.req.clear(); R.seq.clear();
    for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= N - j; ++i) {
            R.req.push_back(-1.0 + 2.0 * i / N);
            R.seq.push_back(-1.0 + 2.0 * j / N);
        }
    Mat Veq;
    dubiner(N, R.req, R.seq, Veq, nullptr, nullptr);
    if (!invert(Veq, R.Veq_inv)) { err = "singular equispaced Vandermonde"; return false; }
    return true;
}

// ---------------------------------------------------------------------------
// Mesh and geometry
// ---------------------------------------------------------------------------
bool build_mesh(const RefOps& R, const MeshSpec& sp, MeshData& D, std::string& err) {
    if (sp.nx < 3 || sp.ny < 3) { err = "nx and ny must be >= 3 (periodic faces must be distinct)"; return false; }
    if (!(sp.x1 > sp.x0) || !(sp.y1 > sp.y0)) { err = "empty domain"; return false; }
    const int nx = sp.nx, ny = sp.ny;
    const long long Kll = 2LL * nx * ny;
    if (Kll > (1LL << 28)) { err = "mesh too large"; return false; }
    const int K = int(Kll);
    D.K = K;
    const double Lx = sp.x1 - sp.x0, Ly = sp.y1 - sp.y0;
    const double xc = 0.5 * (sp.x0 + sp.x1), yc = 0.5 * (sp.y0 + sp.y1);
    const int Np = R.Np, Nq = R.Nq, Nfq = R.Nfq, Nh = R.Nh, Nfp = R.Nfp;
    std::vector<double> VX(3 * size_t(K)), VY(3 * size_t(K));
    std::vector<int> PV(3 * size_t(K));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int q = j * nx + i;
            int tri[2][3][2] = {{{i, j}, {i + 1, j}, {i + 1, j + 1}}, {{i, j}, {i + 1, j + 1}, {i, j + 1}}};
            for (int t = 0; t < 2; ++t) {
                int e = 2 * q + t;
                for (int v = 0; v < 3; ++v) {
                    int ii = tri[t][v][0], jj = tri[t][v][1];
                    VX[3 * e + v] = sp.x0 + Lx * ii / nx;
                    VY[3 * e + v] = sp.y0 + Ly * jj / ny;
                    // periodic: wrapped vertex ids; walls: one id per grid vertex
                    PV[3 * e + v] = sp.walls ? jj * (nx + 1) + ii : (jj % ny) * nx + (ii % nx);
                }
            }
        }
    // face matching by (periodic) vertex pairs; with walls, a boundary face
    // has no partner and is marked 4 e + 3 (its own element, face slot 3)
    D.nbr.assign(3 * size_t(K), -1);
    {
        std::map<std::pair<int, int>, std::vector<int>> faces;
        const int fv[3][2] = {{0, 1}, {1, 2}, {2, 0}};
        for (int e = 0; e < K; ++e)
            for (int f = 0; f < 3; ++f) {
                int a = PV[3 * e + fv[f][0]], b = PV[3 * e + fv[f][1]];
                faces[{std::min(a, b), std::max(a, b)}].push_back(4 * e + f);
            }
        for (auto& kv : faces) {
            if (sp.walls && kv.second.size() == 1) {
                const int a = kv.second[0];
                D.nbr[3 * (a >> 2) + (a & 3)] = 4 * (a >> 2) + 3;
                continue;
            }
            if (kv.second.size() != 2) { err = "a face is not shared by exactly two elements"; return false; }
            int a = kv.second[0], b = kv.second[1];
            D.nbr[3 * (a >> 2) + (a & 3)] = b;
            D.nbr[3 * (b >> 2) + (b & 3)] = a;
        }
    }
    // curved map: warp the equispaced nodes of each affine element
    D.xeq.resize(size_t(K) * Np);
    D.yeq.resize(size_t(K) * Np);
    const double PI = 3.14159265358979323846;
    for (int e = 0; e < K; ++e)
        for (int n = 0; n < Np; ++n) {
            double r = R.req[n], s = R.seq[n];
            double x = -0.5 * (r + s) * VX[3 * e] + 0.5 * (1 + r) * VX[3 * e + 1] + 0.5 * (1 + s) * VX[3 * e + 2];
            double y = -0.5 * (r + s) * VY[3 * e] + 0.5 * (1 + r) * VY[3 * e + 1] + 0.5 * (1 + s) * VY[3 * e + 2];
            double xi = 2.0 * (x - xc) / Lx, eta = 2.0 * (y - yc) / Ly;
            D.xeq[size_t(e) * Np + n] = x + sp.ax * 0.5 * Lx * std::cos(0.5 * PI * xi) * std::cos(1.5 * PI * eta);
            D.yeq[size_t(e) * Np + n] = y + sp.ay * 0.5 * Ly * std::sin(2.0 * PI * xi) * std::cos(0.5 * PI * eta);
        }
    // geometric factors at the hybrid nodes (J-scaled metrics, Sec. 2.7)
    D.geo.assign(size_t(K) * Nh * 4, 0.0);
    D.Jq.assign(size_t(K) * Nq, 0.0);
    D.xq.assign(size_t(K) * Nq, 0.0);
    D.yq.assign(size_t(K) * Nq, 0.0);
    D.xf.assign(size_t(K) * Nfq, 0.0);
    D.yf.assign(size_t(K) * Nfq, 0.0);
    D.minv.assign(size_t(K) * (Np * (Np + 1) / 2), 0.0);
    // per-element geometry and inverse mass matrices, in parallel over elements
    std::atomic<int> bad(0);  // 1: non-positive J at a volume node, 2: at a face node, 3: singular M_h
    auto work = [&](int e_begin, int e_end) {
        std::vector<double> xm(Np), ym(Np);
        Mat Mh(Np, Np), Mhi;
        for (int e = e_begin; e < e_end && !bad.load(std::memory_order_relaxed); ++e) {
            for (int n = 0; n < Np; ++n) {
                double sx = 0, sy = 0;
                for (int m = 0; m < Np; ++m) {
                    sx += R.Veq_inv(n, m) * D.xeq[size_t(e) * Np + m];
                    sy += R.Veq_inv(n, m) * D.yeq[size_t(e) * Np + m];
                }
                xm[n] = sx;
                ym[n] = sy;
            }
            auto eval = [&](const Mat& V, const Mat& Vr, const Mat& Vs, int p, double* out) {
                double x = 0, y = 0, xr = 0, xs = 0, yr = 0, ys = 0;
                for (int n = 0; n < Np; ++n) {
                    x += V(p, n) * xm[n]; y += V(p, n) * ym[n];
                    xr += Vr(p, n) * xm[n]; xs += Vs(p, n) * xm[n];
                    yr += Vr(p, n) * ym[n]; ys += Vs(p, n) * ym[n];
                }
                out[0] = x; out[1] = y;
                out[2] = ys; out[3] = -yr; out[4] = -xs; out[5] = xr;   // rxJ sxJ ryJ syJ
                out[6] = xr * ys - xs * yr;                              // J
            };
            double g7[7];
            for (int q = 0; q < Nq; ++q) {
                eval(R.Vq, R.Vqr, R.Vqs, q, g7);
                if (!(g7[6] > 0.0)) { bad = 1; return; }
                D.xq[size_t(e) * Nq + q] = g7[0];
                D.yq[size_t(e) * Nq + q] = g7[1];
                for (int c = 0; c < 4; ++c) D.geo[(size_t(e) * Nh + q) * 4 + c] = g7[2 + c];
                D.Jq[size_t(e) * Nq + q] = g7[6];
            }
            for (int f = 0; f < Nfq; ++f) {
                eval(R.Vf, R.Vfr, R.Vfs, f, g7);
                if (!(g7[6] > 0.0)) { bad = 2; return; }
                D.xf[size_t(e) * Nfq + f] = g7[0];
                D.yf[size_t(e) * Nfq + f] = g7[1];
                for (int c = 0; c < 4; ++c) D.geo[(size_t(e) * Nh + Nq + f) * 4 + c] = g7[2 + c];
            }
            size_t o = size_t(e) * (Np * (Np + 1) / 2);
            if (sp.wadg) {
                // weight-adjusted inverse M^{-1} M_{1/J} M^{-1} (Sec. 2.8's
                // alternative), with the reference mass matrix M = I of the
                // orthonormal basis under these rules (exact to 2N)
                for (int i = 0; i < Np; ++i)
                    for (int j = 0; j <= i; ++j) {
                        double s = 0;
                        for (int q = 0; q < Nq; ++q) s += R.Vq(q, i) * R.wq[q] / D.Jq[size_t(e) * Nq + q] * R.Vq(q, j);
                        D.minv[o + i * (i + 1) / 2 + j] = s;
                    }
                continue;
            }
            // M_h^k = Vq^T W J Vq and its inverse (Sec. 2.7), packed lower triangle
            for (int i = 0; i < Np; ++i)
                for (int j = 0; j < Np; ++j) {
                    double s = 0;
                    for (int q = 0; q < Nq; ++q) s += R.Vq(q, i) * R.wq[q] * D.Jq[size_t(e) * Nq + q] * R.Vq(q, j);
                    Mh(i, j) = s;
                }
            if (!invert(Mh, Mhi)) { bad = 3; return; }
            for (int i = 0; i < Np; ++i)
                for (int j = 0; j <= i; ++j) D.minv[o + i * (i + 1) / 2 + j] = 0.5 * (Mhi(i, j) + Mhi(j, i));
        }
    };
    const int nthreads = std::max(1, std::min<int>(int(std::thread::hardware_concurrency()), (K + 4095) / 4096));
    if (nthreads == 1) {
        work(0, K);
    } else {
        std::vector<std::thread> pool;
        const int chunk = (K + nthreads - 1) / nthreads;
        for (int t = 0; t < nthreads; ++t) {
            const int b0 = t * chunk, b1 = std::min(K, b0 + chunk);
            if (b0 < b1) pool.emplace_back(work, b0, b1);
        }
        for (auto& th : pool) th.join();
    }
    if (bad == 1) { err = "non-positive Jacobian at a volume node"; return false; }
    if (bad == 2) { err = "non-positive Jacobian at a face node"; return false; }
    if (bad == 3) { err = "singular curved mass matrix"; return false; }
    // every face node must meet its partner (reversed order) modulo the period
    const double tol = 1e-9 * std::min(Lx / nx, Ly / ny);
    for (int e = 0; e < K; ++e)
        for (int f = 0; f < 3; ++f) {
            int nb = D.nbr[3 * e + f];
            int en = nb >> 2, fn = nb & 3;
            if (fn == 3) continue;  // wall
            for (int i = 0; i < Nfp; ++i) {
                int a = e * Nfq + f * Nfp + i;
                int b = en * Nfq + fn * Nfp + (Nfp - 1 - i);
                double dx = D.xf[b] - D.xf[a], dy = D.yf[b] - D.yf[a];
                dx -= Lx * std::round(dx / Lx);
                dy -= Ly * std::round(dy / Ly);
                if (std::fabs(dx) > tol || std::fabs(dy) > tol) {
                    err = "face quadrature nodes of neighbouring elements do not match";
                    return false;
                }
            }
        }
    return true;
}

}  // namespace esdg
