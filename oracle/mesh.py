"""Structured periodic triangulation, curved warp and geometric factors
(oracle; test infrastructure only).  Follows Sec. 2.7 (J^k, G^k_ij, B^{i,k},
M_h^k) and the mesh warping of Sec. 4.

Readings (the paper is silent on these):
  * mesh: an nx x ny grid of quadrilaterals on [x0,x1] x [y0,y1], periodic in
    both directions; quad (i, j) splits along its lower-left to upper-right
    diagonal into element 2q = (v(i,j), v(i+1,j), v(i+1,j+1)) and element
    2q+1 = (v(i,j), v(i+1,j+1), v(i,j+1)), q = j*nx + i, both counter-
    clockwise.  Reference vertices v1=(-1,-1), v2=(1,-1), v3=(-1,1) map to
    the element's vertices in that order.
  * curved elements: the warp is applied to the degree-N equispaced nodes of
    each affine element and the map is their degree-N interpolant (C0 across
    shared edges).  Warp, with xi = 2(x-xc)/Lx, eta = 2(y-yc)/Ly:
        x += ax * Lx/2 * cos(pi xi / 2) cos(3 pi eta / 2)
        y += ay * Ly/2 * sin(2 pi xi)   cos(pi eta / 2)
    which vanishes on the domain boundary, so periodic faces still match.
  * G^k_ij of Sec. 2.7 is used J-scaled (rxJ = J dr/dx, ...), which is what
    pairs with the J-weighted mass matrix M_h^k = Vq^T W J Vq.
  * mass="weight_adjusted" replaces the stored inverse (M_h^k)^{-1} by the
    weight-adjusted inverse that Sec. 2.8 names as the way to avoid storing
    it: M^{-1} M_{1/J} M^{-1}, with the reference mass matrix M = Vq^T W Vq and
    M_{1/J} = Vq^T W diag(1/J^k) Vq (the weight-adjusted approximation of
    Chan, Hewett and Warburton, 2017).  It equals (M_h^k)^{-1} when J^k is
    constant (affine elements).
"""

import numpy as np

from .refelem import basis


class Mesh:
    """Mesh, connectivity and geometric factors at the hybrid nodes.

    Geometric arrays are (K, Nh) over the Nq volume then Nfq face nodes:
    rxJ, sxJ, ryJ, syJ, J.  Face arrays are (K, Nfq): nxJ, nyJ, sJ.
    mapP (K*Nfq,) gives, for every face node, the flat index of the matching
    face node on the neighbouring element (periodic wrap included).  With
    walls=True the four sides are reflective walls (Sec. 2.9): a boundary face
    has no partner, its nodes map to themselves and wall (K, 3) marks it.
    """

    def __init__(self, ref, nx, ny, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, ax=0.0, ay=0.0, walls=False,
                 mass="exact"):
        if mass not in ("exact", "weight_adjusted"):
            raise ValueError(mass)
        self.ref = ref
        self.walls = walls
        self.mass = mass
        self.nx, self.ny = nx, ny
        self.x0, self.x1, self.y0, self.y1 = x0, x1, y0, y1
        self.Lx, self.Ly = x1 - x0, y1 - y0
        self.ax, self.ay = ax, ay
        self.K = 2 * nx * ny
        self.dx = self.Lx / nx
        self._build_elements()
        self._build_nodes()
        self._build_geometry()
        self._build_connectivity()

    # -- topology ----------------------------------------------------------
    def _build_elements(self):
        nx, ny = self.nx, self.ny
        vx = lambda i: self.x0 + self.Lx * i / nx  # noqa: E731
        vy = lambda j: self.y0 + self.Ly * j / ny  # noqa: E731
        K = self.K
        self.VX = np.zeros((K, 3))
        self.VY = np.zeros((K, 3))
        self.EToPV = np.zeros((K, 3), dtype=np.int64)  # periodic vertex ids
        if self.walls:
            pv = lambda i, j: j * (nx + 1) + i  # noqa: E731
        else:
            pv = lambda i, j: (j % ny) * nx + (i % nx)  # noqa: E731
        for j in range(ny):
            for i in range(nx):
                q = j * nx + i
                tris = [((i, j), (i + 1, j), (i + 1, j + 1)),
                        ((i, j), (i + 1, j + 1), (i, j + 1))]
                for t, tri in enumerate(tris):
                    e = 2 * q + t
                    for v, (ii, jj) in enumerate(tri):
                        self.VX[e, v] = vx(ii)
                        self.VY[e, v] = vy(jj)
                        self.EToPV[e, v] = pv(ii, jj)

    def affine_map(self, r, s):
        """x = -(r+s)/2 v1 + (1+r)/2 v2 + (1+s)/2 v3 per element; (K, npts)."""
        r = np.asarray(r)[None, :]
        s = np.asarray(s)[None, :]
        X, Y = self.VX, self.VY
        x = -0.5 * (r + s) * X[:, 0:1] + 0.5 * (1 + r) * X[:, 1:2] + 0.5 * (1 + s) * X[:, 2:3]
        y = -0.5 * (r + s) * Y[:, 0:1] + 0.5 * (1 + r) * Y[:, 1:2] + 0.5 * (1 + s) * Y[:, 2:3]
        return x, y

    def warp(self, x, y):
        """Curving map of the domain (reading in the module docstring)."""
        xc = 0.5 * (self.x0 + self.x1)
        yc = 0.5 * (self.y0 + self.y1)
        xi = 2.0 * (x - xc) / self.Lx
        eta = 2.0 * (y - yc) / self.Ly
        xw = x + self.ax * 0.5 * self.Lx * np.cos(0.5 * np.pi * xi) * np.cos(1.5 * np.pi * eta)
        yw = y + self.ay * 0.5 * self.Ly * np.sin(2.0 * np.pi * xi) * np.cos(0.5 * np.pi * eta)
        return xw, yw

    # -- nodes ---------------------------------------------------------------
    def _build_nodes(self):
        ref = self.ref
        # physical positions of the degree-N equispaced nodes (curved map data)
        xe, ye = self.affine_map(ref.req, ref.seq)
        self.xeq, self.yeq = self.warp(xe, ye)
        # modal coefficients of the map x(r,s), y(r,s)
        Veq_inv = np.linalg.inv(ref.Veq)
        self.xmodal = self.xeq @ Veq_inv.T
        self.ymodal = self.yeq @ Veq_inv.T

    def map_points(self, r, s):
        V = basis(self.ref.N, np.asarray(r), np.asarray(s))
        return self.xmodal @ V.T, self.ymodal @ V.T

    # -- geometry (Sec. 2.7) ----------------------------------------------------
    def _metrics_at(self, Vr, Vs):
        xr = self.xmodal @ Vr.T
        xs = self.xmodal @ Vs.T
        yr = self.ymodal @ Vr.T
        ys = self.ymodal @ Vs.T
        J = xr * ys - xs * yr
        return ys, -yr, -xs, xr, J  # rxJ, sxJ, ryJ, syJ, J

    def _build_geometry(self):
        ref = self.ref
        rxq, sxq, ryq, syq, Jq = self._metrics_at(ref.Vqr, ref.Vqs)
        rxf, sxf, ryf, syf, Jf = self._metrics_at(ref.Vfr, ref.Vfs)
        self.rxJ = np.hstack([rxq, rxf])
        self.sxJ = np.hstack([sxq, sxf])
        self.ryJ = np.hstack([ryq, ryf])
        self.syJ = np.hstack([syq, syf])
        self.Jq = Jq
        self.Jh = np.hstack([Jq, Jf])
        if np.any(Jq <= 0):
            raise ValueError("non-positive Jacobian")
        # physical scaled normals B^{i,k} = W_f diag(nJ_i), nJ_i = sum_j G_ij n-hat_j
        self.nxJ = rxf * ref.nr[None, :] + sxf * ref.ns[None, :]
        self.nyJ = ryf * ref.nr[None, :] + syf * ref.ns[None, :]
        self.sJ = np.sqrt(self.nxJ ** 2 + self.nyJ ** 2)
        # quadrature point coordinates
        self.xq, self.yq = self.map_points(ref.rq, ref.sq)
        self.xf, self.yf = self.map_points(ref.rf, ref.sf)
        # curved mass matrices M_h^k = Vq^T W J^k Vq and their inverses (Sec. 2.7)
        VqW = ref.Vq * ref.w[:, None]
        self.Mh = np.einsum("qn,kq,qm->knm", VqW, Jq, ref.Vq)
        if self.mass == "exact":
            self.Mh_inv = np.linalg.inv(self.Mh)
        else:
            # weight-adjusted inverse M^{-1} M_{1/J} M^{-1} (Sec. 2.8's remedy)
            M_ref_inv = np.linalg.inv(VqW.T @ ref.Vq)
            M_invJ = np.einsum("qn,kq,qm->knm", VqW, 1.0 / Jq, ref.Vq)
            self.Mh_inv = M_ref_inv[None] @ M_invJ @ M_ref_inv[None]

    # -- connectivity ------------------------------------------------------------
    def _build_connectivity(self):
        """Match faces by their periodic vertex pair, then face nodes in
        reverse order (two counter-clockwise elements run a shared edge in
        opposite directions)."""
        K = self.K
        fv = [(0, 1), (1, 2), (2, 0)]
        table = {}
        for e in range(K):
            for f, (a, b) in enumerate(fv):
                key = tuple(sorted((self.EToPV[e, a], self.EToPV[e, b])))
                table.setdefault(key, []).append((e, f))
        self.EToE = np.zeros((K, 3), dtype=np.int64)
        self.EToF = np.zeros((K, 3), dtype=np.int64)
        self.wall = np.zeros((K, 3), dtype=bool)
        for key, lst in table.items():
            if self.walls and len(lst) == 1:
                (e1, f1), = lst
                self.EToE[e1, f1], self.EToF[e1, f1] = e1, f1
                self.wall[e1, f1] = True
                continue
            if len(lst) != 2:
                raise ValueError("face %s is shared by %d elements" % (key, len(lst)))
            (e1, f1), (e2, f2) = lst
            self.EToE[e1, f1], self.EToF[e1, f1] = e2, f2
            self.EToE[e2, f2], self.EToF[e2, f2] = e1, f1
        Nfp = self.ref.N + 1
        Nfq = 3 * Nfp
        mapP = np.zeros(K * Nfq, dtype=np.int64)
        for e in range(K):
            for f in range(3):
                en, fn = self.EToE[e, f], self.EToF[e, f]
                for i in range(Nfp):
                    if self.wall[e, f]:
                        mapP[e * Nfq + f * Nfp + i] = e * Nfq + f * Nfp + i
                    else:
                        mapP[e * Nfq + f * Nfp + i] = en * Nfq + fn * Nfp + (Nfp - 1 - i)
        self.mapP = mapP
