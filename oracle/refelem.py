"""Reference-element operators (oracle; test infrastructure only).

Follows Sec. 2.1 (P^N, V_q, V_f, W, W_f, D^i, M, P_q), Sec. 2.2 (Q-hat^i, B^i,
Q^i, E, V_h, SBP property eq. (SBP_Q)) and Sec. 2.3 (hybridized Q_h^i,
Theorem 2.1) of the paper.

Readings (the paper leaves these open, Sec. 2.1):
  * basis: the orthonormal Dubiner (Koornwinder) basis, built from Jacobi
    polynomials through the collapsed map a = 2(1+r)/(1-s) - 1, b = s.
    Mode order: for i = 0..N, for j = 0..N-i.
  * volume quadrature: the collapsed (Stroud conical) product rule with N+1
    Gauss-Legendre points in a and N+1 Gauss-Jacobi(1,0) points in b,
    exact to degree 2N+1 (the paper asks for at least 2N-1).
  * surface quadrature: N+1 Gauss-Legendre points on each face (exact to
    degree 2N+1 on faces; the paper asks for at least 2N).
  * faces: f1 v1->v2 (s=-1), f2 v2->v3 (r+s=0), f3 v3->v1 (r=-1) with
    reference vertices v1=(-1,-1), v2=(1,-1), v3=(-1,1).  W_f holds the
    Gauss-Legendre weights of the face parameter t in [-1,1]; the reference
    normals n-hat are the outward normals scaled by the face Jacobian
    (Sec. 2.1), so B^i = W_f diag(n-hat_i) carries the face measure once.

Jacobi polynomials and Gauss rules come from scipy.special (library
primitives used as single steps).
"""

import numpy as np
from scipy import special


# ---------------------------------------------------------------------------
# 1D orthonormal Jacobi polynomials and Gauss rules
# ---------------------------------------------------------------------------

def _jacobi_norm(n, alpha, beta):
    """Squared L2 norm of the classical Jacobi polynomial P_n^(alpha,beta)
    under the weight (1-x)^alpha (1+x)^beta on [-1, 1]."""
    return (2.0 ** (alpha + beta + 1) / (2 * n + alpha + beta + 1)
            * special.gamma(n + alpha + 1) * special.gamma(n + beta + 1)
            / (special.gamma(n + alpha + beta + 1) * special.gamma(n + 1)))


def jacobi(x, alpha, beta, n):
    """Orthonormal Jacobi polynomial of degree n at x."""
    return special.eval_jacobi(n, alpha, beta, x) / np.sqrt(_jacobi_norm(n, alpha, beta))


def jacobi_deriv(x, alpha, beta, n):
    """d/dx of the orthonormal Jacobi polynomial of degree n at x, from
    d/dx P_n^(a,b) = (n+a+b+1)/2 * P_{n-1}^(a+1,b+1)."""
    x = np.asarray(x, dtype=np.float64)
    if n == 0:
        return np.zeros_like(x)
    dp = 0.5 * (n + alpha + beta + 1) * special.eval_jacobi(n - 1, alpha + 1, beta + 1, x)
    return dp / np.sqrt(_jacobi_norm(n, alpha, beta))


def gauss_legendre(n):
    x, w = special.roots_legendre(n)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


def gauss_jacobi(n, alpha, beta):
    x, w = special.roots_jacobi(n, alpha, beta)
    return np.asarray(x, np.float64), np.asarray(w, np.float64)


# ---------------------------------------------------------------------------
# Reference triangle
# ---------------------------------------------------------------------------

def rs_to_ab(r, s):
    """Collapsed coordinates of the reference triangle; a is set to -1 at the
    top vertex s = 1 where it is undefined (every mode with i > 0 vanishes
    there, and the i = 0 modes do not depend on a)."""
    r = np.asarray(r, np.float64)
    s = np.asarray(s, np.float64)
    a = np.full_like(r, -1.0)
    ok = np.abs(1.0 - s) > 1e-14
    a[ok] = 2.0 * (1.0 + r[ok]) / (1.0 - s[ok]) - 1.0
    return a, s.copy()


def mode_list(N):
    return [(i, j) for i in range(N + 1) for j in range(N + 1 - i)]


def num_modes(N):
    return (N + 1) * (N + 2) // 2


def basis(N, r, s, derivs=False):
    """Orthonormal Dubiner basis phi_{ij} = sqrt(2) P_i(a) P_j^(2i+1,0)(b) (1-b)^i
    at points (r, s) (Sec. 2.1: some basis of P^N; reading above).

    Returns V (npts x Np) and, if derivs, Vr = d phi/dr and Vs = d phi/ds from
    the chain rule d/dr = 2/(1-b) d/da, d/ds = (1+a)/(1-b) d/da + d/db.
    """
    a, b = rs_to_ab(r, s)
    modes = mode_list(N)
    V = np.zeros((a.size, len(modes)))
    Vr = np.zeros_like(V)
    Vs = np.zeros_like(V)
    if derivs and np.any(np.abs(1.0 - b) < 1e-12):
        raise ValueError("basis derivatives are not evaluated at the vertex s = 1")
    for n, (i, j) in enumerate(modes):
        fa = jacobi(a, 0, 0, i)
        gb = jacobi(b, 2 * i + 1, 0, j)
        V[:, n] = np.sqrt(2.0) * fa * gb * (1.0 - b) ** i
        if not derivs:
            continue
        dfa = jacobi_deriv(a, 0, 0, i)
        dgb = jacobi_deriv(b, 2 * i + 1, 0, j)
        # d phi / da and d phi / db
        if i > 0:
            pa = np.sqrt(2.0) * dfa * gb * (1.0 - b) ** i
            pb = np.sqrt(2.0) * fa * (dgb * (1.0 - b) ** i - i * gb * (1.0 - b) ** (i - 1))
        else:
            pa = np.zeros_like(a)
            pb = np.sqrt(2.0) * fa * dgb
        Vr[:, n] = pa * 2.0 / (1.0 - b)
        Vs[:, n] = pa * (1.0 + a) / (1.0 - b) + pb
    if derivs:
        return V, Vr, Vs
    return V


def triangle_quadrature(n1d):
    """Collapsed product rule with n1d points per direction, exact for
    polynomials of total degree 2*n1d - 1 on the reference triangle.
    int_T f dr ds = int int f(r(a,b), b) (1-b)/2 da db."""
    xa, wa = gauss_legendre(n1d)
    xb, wb = gauss_jacobi(n1d, 1.0, 0.0)
    A, B = np.meshgrid(xa, xb, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    r = 0.5 * (1.0 + A) * (1.0 - B) - 1.0
    s = B
    w = 0.5 * WA * WB
    return r.ravel(), s.ravel(), w.ravel()


def face_quadrature(N):
    """N+1 Gauss-Legendre points on each face, faces in the order f1, f2, f3.

    Returns (rf, sf, wf, nr, ns): nodes, Gauss-Legendre weights of the face
    parameter, and the outward reference normal scaled by the face Jacobian
    (f1: (0,-1), f2: (1,1) = sqrt(2) * unit normal, f3: (-1,0))."""
    t, w = gauss_legendre(N + 1)
    one = np.ones_like(t)
    rf = np.concatenate([t, -t, -one])
    sf = np.concatenate([-one, t, -t])
    wf = np.concatenate([w, w, w])
    nr = np.concatenate([0 * one, one, -one])
    ns = np.concatenate([-one, one, 0 * one])
    return rf, sf, wf, nr, ns


def equispaced_nodes(N):
    """Degree-N equispaced nodes of the reference triangle, s-major:
    for j = 0..N (s), for i = 0..N-j (r).  They contain the vertices and
    N-1 interior points per edge."""
    r, s = [], []
    for j in range(N + 1):
        for i in range(N + 1 - j):
            r.append(-1.0 + 2.0 * i / N)
            s.append(-1.0 + 2.0 * j / N)
    return np.array(r), np.array(s)


class RefElem:
    """All reference-element matrices of Sec. 2.1-2.3 for degree N.

    Attributes (shapes): Vq (Nq,Np), Vf (Nfq,Np), w (Nq,), wf (Nfq,),
    M, Pq (Np,Nq), Dr/Ds (Np,Np), Qr_hat/Qs_hat (Np,Np), Br/Bs (Nfq,Nfq),
    Qr/Qs (Nq,Nq), E (Nfq,Nq), Vh (Nh,Np), Qhr/Qhs (Nh,Nh),
    Veq (Np,Np) Vandermonde at the equispaced nodes, and the error rule
    (rq2, sq2, wq2, Vq2) exact to degree 2N+3 (>= 2N+2, Sec. 4.1).
    """

    def __init__(self, N):
        if N < 1:
            raise ValueError("N >= 1")
        self.N = N
        self.Np = num_modes(N)
        # volume and surface quadrature (Sec. 2.1)
        self.rq, self.sq, self.w = triangle_quadrature(N + 1)
        self.rf, self.sf, self.wf, self.nr, self.ns = face_quadrature(N)
        self.Nq = self.rq.size
        self.Nfq = self.rf.size
        self.Nh = self.Nq + self.Nfq
        self.Vq, self.Vqr, self.Vqs = basis(N, self.rq, self.sq, derivs=True)
        self.Vf, self.Vfr, self.Vfs = basis(N, self.rf, self.sf, derivs=True)
        W = np.diag(self.w)
        Wf = np.diag(self.wf)
        # mass matrix and quadrature L2 projection (Sec. 2.1, eq. (PqVq))
        self.M = self.Vq.T @ W @ self.Vq
        self.Pq = np.linalg.solve(self.M, self.Vq.T @ W)
        # modal differentiation: coefficients of d/dr of a degree-N polynomial
        # (Sec. 2.1); derivatives lie in P^{N-1}, so projecting their
        # quadrature values recovers them exactly.
        self.Dr = self.Pq @ self.Vqr
        self.Ds = self.Pq @ self.Vqs
        # Q-hat^i = M D^i, B^i = W_f diag(n-hat_i) (Sec. 2.2)
        self.Qr_hat = self.M @ self.Dr
        self.Qs_hat = self.M @ self.Ds
        self.Br = Wf @ np.diag(self.nr)
        self.Bs = Wf @ np.diag(self.ns)
        # nodal operators at volume quadrature points (Sec. 2.2)
        self.Qr = self.Pq.T @ self.Qr_hat @ self.Pq
        self.Qs = self.Pq.T @ self.Qs_hat @ self.Pq
        self.E = self.Vf @ self.Pq
        self.Vh = np.vstack([self.Vq, self.Vf])
        # hybridized operators (Sec. 2.3)
        self.Qhr = self._hybridize(self.Qr, self.Br)
        self.Qhs = self._hybridize(self.Qs, self.Bs)
        Z = np.zeros((self.Nq, self.Nq))
        self.Bhr = np.block([[Z, np.zeros((self.Nq, self.Nfq))],
                             [np.zeros((self.Nfq, self.Nq)), self.Br]])
        self.Bhs = np.block([[Z, np.zeros((self.Nq, self.Nfq))],
                             [np.zeros((self.Nfq, self.Nq)), self.Bs]])
        # equispaced nodes for the curved map and the C0 bathymetry (Sec. 4, 4.1)
        self.req, self.seq = equispaced_nodes(N)
        self.Veq = basis(N, self.req, self.seq)
        # error quadrature, exact to degree >= 2N+2 (Sec. 4.1)
        self.rq2, self.sq2, self.wq2 = triangle_quadrature(N + 2)
        self.Vq2 = basis(N, self.rq2, self.sq2)

    def _hybridize(self, Q, B):
        """Q_h = 1/2 [[Q - Q^T, E^T B], [-B E, B]] (Sec. 2.3)."""
        E = self.E
        return 0.5 * np.block([[Q - Q.T, E.T @ B], [-B @ E, B]])
