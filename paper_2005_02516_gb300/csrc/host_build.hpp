// Host-side (FP64) construction of the reference-element operators, the
// structured periodic curved mesh and its geometric factors for the ESDG
// shallow-water scheme (Wu, Kubatko, Chan, arXiv 2005.02516, Sec. 2.1-2.3 and
// Sec. 2.7).  Everything here runs once at set-up; the per-stage work runs in
// the CUDA kernels.
#pragma once

#include <string>
#include <vector>

namespace esdg {

// Dense row-major matrix of doubles.
struct Mat {
    int r = 0, c = 0;
    std::vector<double> a;
    Mat() = default;
    Mat(int r_, int c_) : r(r_), c(c_), a(size_t(r_) * c_, 0.0) {}
    double& operator()(int i, int j) { return a[size_t(i) * c + j]; }
    double operator()(int i, int j) const { return a[size_t(i) * c + j]; }
};

Mat matmul(const Mat& A, const Mat& B);
Mat transpose(const Mat& A);
bool invert(const Mat& A, Mat& Ainv);  // Gauss-Jordan with partial pivoting

// Reference element of degree N.
struct RefOps {
    int N = 0, Np = 0, Nq = 0, Nfp = 0, Nfq = 0, Nh = 0;
    std::vector<double> rq, sq, wq;        // volume rule
    std::vector<double> rf, sf, wf;        // face rule (faces f1, f2, f3)
    std::vector<double> nr, ns;            // scaled reference normals at face nodes
    std::vector<double> req, seq;          // equispaced nodes
    Mat Vq, Vf, Vqr, Vqs, Vfr, Vfs;        // basis and its gradients at the rules
    Mat Pq;                                // (Np x Nq) quadrature L2 projection
    Mat Vh;                                // (Nh x Np)
    Mat Qsr, Qss;                          // skew hybridized operators Q_h - Q_h^T (Nh x Nh)
    Mat Veq_inv;                           // inverse Vandermonde at the equispaced nodes
    std::vector<int> fmap;                 // SBP rule only: volume node of each face node (I_f)
};

// rule 0: collapsed Gauss rule, (N+1)^2 points, exact to 2N+1;
// rule 1: fully symmetric rule exact to 2N (3, 6, 12, 16, 25 points);
// rule 2: SBP rule of Sec. 3.1, exact to 2N-1 with the face Gauss-Legendre
//         points among its nodes (6, 10, 18, 22, 34 points).
bool build_reference(int N, int rule, RefOps& ref, std::string& err);
bool symmetric_rule(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w, std::string& err);
bool sbp_rule(int N, std::vector<double>& r, std::vector<double>& s, std::vector<double>& w, std::string& err);

// Orthonormal Dubiner basis and (optionally) its gradients at points (r, s).
void dubiner(int N, const std::vector<double>& r, const std::vector<double>& s,
             Mat& V, Mat* Vr, Mat* Vs);

struct MeshSpec {
    int nx, ny;
    double x0, x1, y0, y1;
    double ax, ay;
    bool walls;  // reflective walls on the four sides instead of periodic wrap
    bool wadg;   // minv holds the weight-adjusted inverse Vq^T W diag(1/J) Vq instead of (M_h^k)^{-1}
};

// Mesh, connectivity and geometry.  Per-element arrays are [K][...].
struct MeshData {
    int K = 0;
    std::vector<double> xeq, yeq;   // [K][Np] equispaced node positions (curved)
    std::vector<double> xq, yq;     // [K][Nq]
    std::vector<double> xf, yf;     // [K][Nfq]
    std::vector<double> geo;        // [K][Nh][4]: rxJ, sxJ, ryJ, syJ
    std::vector<double> Jq;         // [K][Nq]
    std::vector<double> minv;       // [K][Np(Np+1)/2] packed lower triangle of (M_h^k)^-1
                                    // (or of its weight-adjusted approximation, MeshSpec::wadg)
    std::vector<int> nbr;           // [K][3]: 4 * neighbour element + neighbour face (4 e + 3: wall)
};

bool build_mesh(const RefOps& ref, const MeshSpec& spec, MeshData& mesh, std::string& err);

}  // namespace esdg
