"""Semi-discrete ESDG right-hand side and LSRK45 time stepping (oracle; test
infrastructure only).

The right-hand side is eq. (dgform) of Sec. 2.8 written out literally, one
dense hybridized operator per element:

  M_h^k du/dt = - sum_{i=x,y} V_h^T (2 Q_h^{i,k} o F^i) 1
                - sum_{i=x,y} V_f^T B^{i,k} (f_S^i(u~+, u~_f) - f^i(u~_f))
                + V_f^T W_f (1/2 lambda sJ (u~+ - u~_f))          [LF, Sec. 2.8]
                + S                                                  [source]
                + V_q^T W J f(x_q, t)                                [forcing]

with u~ the entropy-projected conservative variables of Sec. 2.6,
Q_h^{i,k}[l,m] = 1/2 sum_j Q_h^j[l,m] (G_ij[l] + G_ij[m]) (Sec. 2.7) and
(F^i)_{lm} = f_S^i(u~_l, u~_m).

Readings:
  * the entropy projection on curved elements is J-weighted,
    v_h = (M_h^k)^{-1} V_q^T W J v(u_q): the entropy argument of Theorem 2.2
    pairs v_h with M_h^k du/dt, which equals 1^T W J dS/dt only for this
    weighting (Sec. 2.6 prints the affine P_q).
  * the source S = -g V_h^T [0; diag(h~) Q_h^{x,k} b_h; diag(h~) Q_h^{y,k} b_h]
    lives on the hybrid nodes and uses the same operator as the flux
    differencing, which is what the well-balancing argument of Theorem 2.2
    uses (Sec. 2.8 prints diag(h) Q b without naming the nodes).
  * Lax-Friedrichs: lambda = max over both sides of |u.n| + sqrt(g h) on the
    entropy-projected states, penalty on the jump of u~ (Sec. 2.8, Sec. 4).
  * time step dt = CFL h / C_N, C_N = (N+1)(N+2)/2 (Sec. 4), with h the quad
    spacing of the structured grid (the paper does not define h).
  * mass="weight_adjusted": every (M_h^k)^{-1} above, in the projection and in
    the update alike, is the weight-adjusted inverse of mesh.py (Sec. 2.8's
    named alternative to storing the inverses).  Using the same matrix in both
    places keeps the entropy identity of Theorem 2.2 exact; the projection
    then reproduces constants only where J^k is constant, so on curved
    elements a lake at rest is preserved only to the accuracy of the
    weight-adjusted approximation, and the conserved mass is sum_k 1^T
    M~_k u_h with M~_k the inverse of the weight-adjusted matrix.
"""

import numpy as np

from . import swe
from .mesh import Mesh
from .refelem import RefElem

# Carpenter & Kennedy (1994) fourth-order, five-stage 2N-storage Runge-Kutta,
# the integrator named in Sec. 4: res = A_s res + dt rhs(u, t + C_s dt); u += B_s res.
LSRK45_A = np.array([0.0,
                     -567301805773.0 / 1357537059087.0,
                     -2404267990393.0 / 2016746695238.0,
                     -3550918686646.0 / 2091501179385.0,
                     -1275806237668.0 / 842570457699.0])
LSRK45_B = np.array([1432997174477.0 / 9575080441755.0,
                     5161836677717.0 / 13612068292357.0,
                     1720146321549.0 / 2090206949498.0,
                     3134564353537.0 / 4481467310338.0,
                     2277821191437.0 / 14882151754819.0])
LSRK45_C = np.array([0.0,
                     1432997174477.0 / 9575080441755.0,
                     2526269341429.0 / 6820363962896.0,
                     2006345519317.0 / 3224310063776.0,
                     2802321613138.0 / 2924317926251.0])


def mms_sine_forcing(x, y, t, g, amp=0.1, bamp=0.1, u0=0.5, v0=0.5):
    """Forcing f = q_t + div F(q) + (0, g h b_x, g h b_y) of the manufactured
    solution h = 2 + amp sin(pi(x+y-t)), u = u0, v = v0, b = bamp cos(pi x) cos(pi y).

    Derived by hand (and checked symbolically in the tests):
      h_t = -amp pi cos(theta), h_x = h_y = amp pi cos(theta), theta = pi(x+y-t)
      f_h  = h_t + u0 h_x + v0 h_y
      f_hu = u0 h_t + (u0^2 + g h) h_x + u0 v0 h_y + g h b_x
      f_hv = v0 h_t + u0 v0 h_x + (v0^2 + g h) h_y + g h b_y
    """
    th = np.pi * (x + y - t)
    h = 2.0 + amp * np.sin(th)
    c = amp * np.pi * np.cos(th)
    ht, hx, hy = -c, c, c
    bx = -bamp * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
    by = -bamp * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
    fh = ht + u0 * hx + v0 * hy
    fhu = u0 * ht + (u0 * u0 + g * h) * hx + u0 * v0 * hy + g * h * bx
    fhv = v0 * ht + u0 * v0 * hx + (v0 * v0 + g * h) * hy + g * h * by
    return np.stack([fh, fhu, fhv])


class Oracle:
    """FP64 ESDG on a structured periodic (optionally curved) triangle mesh.

    State layout: u_h[field, element, mode], fields (h, hu, hv).
    """

    def __init__(self, N, nx, ny, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, ax=0.0, ay=0.0,
                 g=1.0, cfl=0.25, lf=True, forcing=None, rule="collapsed", walls=False, mass="exact"):
        self.ref = RefElem(N, rule)
        self.mesh = Mesh(self.ref, nx, ny, x0, x1, y0, y1, ax, ay, walls=walls, mass=mass)
        self.N, self.K = N, self.mesh.K
        self.g, self.cfl, self.lf = g, cfl, lf
        self.forcing = forcing  # None or callable (x, y, t, g) -> (3, ...)
        ref, mesh = self.ref, self.mesh
        self.Np, self.Nq, self.Nfq, self.Nh = ref.Np, ref.Nq, ref.Nfq, ref.Nh
        self.b_modal = np.zeros((self.K, self.Np))
        self._bathymetry_at_nodes()
        self.Veq_inv = np.linalg.inv(ref.Veq)

    # -- problem data ------------------------------------------------------------
    def points(self, kind):
        """Physical coordinates: 'nodal' (K, Np) equispaced nodes, 'volq' (K, Nq),
        'faceq' (K, Nfq), 'errq' (K, Nq2) of the error rule."""
        m = self.mesh
        if kind == "nodal":
            return m.xeq, m.yeq
        if kind == "volq":
            return m.xq, m.yq
        if kind == "faceq":
            return m.xf, m.yf
        if kind == "errq":
            return m.map_points(self.ref.rq2, self.ref.sq2)
        raise ValueError(kind)

    def set_bathymetry(self, b_nodal):
        """b is interpolated by a degree-N polynomial through its values at
        the equispaced nodes of each element (C0 across elements, Sec. 4.1)."""
        self.b_modal = np.asarray(b_nodal, np.float64) @ self.Veq_inv.T
        self._bathymetry_at_nodes()

    def _bathymetry_at_nodes(self):
        self.bq = self.b_modal @ self.ref.Vq.T
        self.bh = self.b_modal @ self.ref.Vh.T

    def project(self, q_volq):
        """J-weighted L2 projection (M_h^k)^{-1} V_q^T W J q onto P^N
        (Sec. 2.1, Sec. 2.7); q_volq is (..., K, Nq)."""
        ref, m = self.ref, self.mesh
        rhs = np.einsum("qn,kq,...kq->...kn", ref.Vq * ref.w[:, None], m.Jq, q_volq)
        return np.einsum("knm,...km->...kn", m.Mh_inv, rhs)

    def init_state(self, q_volq, surface=False):
        """Project (h, hu, hv) given at volume quadrature points.  With
        surface=True, q_volq[0] holds the free surface H = h + b and the depth
        is set to Pi(H) - b_h so that a lake at rest is exact (Sec. 4.1)."""
        u = self.project(np.asarray(q_volq, np.float64))
        if surface:
            u[0] = u[0] - self.b_modal
        return u

    def dt(self):
        CN = (self.N + 1) * (self.N + 2) / 2.0
        return self.cfl * self.mesh.dx / CN

    # -- entropy projection (Sec. 2.6) ----------------------------------------------
    def entropy_projection(self, u_h):
        """u_q = Vq u_h, v_q = v(u_q), v_h = J-weighted projection of v_q,
        v~ = Vh v_h, u~ = u(v~).  Returns (u~ (3,K,Nh), v_h (3,K,Np))."""
        ref = self.ref
        uq = np.einsum("qn,ckn->ckq", ref.Vq, u_h)
        vq = swe.entropy_vars(uq, self.bq, self.g)
        vh = self.project(vq)
        vt = np.einsum("hn,ckn->ckh", ref.Vh, vh)
        ut = swe.cons_vars(vt, self.bh, self.g)
        return ut, vh

    # -- right-hand side ----------------------------------------------------------
    def rhs(self, u_h, t=0.0, chunk=1024):
        """du_h/dt of eq. (dgform) for every element; (3, K, Np)."""
        ut, _ = self.entropy_projection(u_h)
        out = np.zeros_like(u_h)
        for k0 in range(0, self.K, chunk):
            k1 = min(self.K, k0 + chunk)
            out[:, k0:k1] = self._rhs_rows(ut, np.arange(k0, k1), t)
        return out

    def rhs_elements(self, u_h, elems, t=0.0):
        """du_h/dt on the listed elements only (for sampled comparisons at
        large K): the entropy projection runs on these elements and their
        face neighbours."""
        elems = np.asarray(elems, dtype=np.int64)
        nbr = self.mesh.EToE[elems].ravel()
        need = np.unique(np.concatenate([elems, nbr]))
        ut = np.full((3, self.K, self.Nh), np.nan)
        sub = self._entropy_projection_subset(u_h, need)
        ut[:, need] = sub
        return self._rhs_rows(ut, elems, t)

    def _entropy_projection_subset(self, u_h, ks):
        ref, m = self.ref, self.mesh
        uq = np.einsum("qn,ckn->ckq", ref.Vq, u_h[:, ks])
        vq = swe.entropy_vars(uq, self.bq[ks], self.g)
        rhs = np.einsum("qn,kq,ckq->ckn", ref.Vq * ref.w[:, None], m.Jq[ks], vq)
        vh = np.einsum("knm,ckm->ckn", m.Mh_inv[ks], rhs)
        vt = np.einsum("hn,ckn->ckh", ref.Vh, vh)
        return swe.cons_vars(vt, self.bh[ks], self.g)

    def _rhs_rows(self, ut, ks, t):
        ref, m, g = self.ref, self.mesh, self.g
        Nq, Nfq = self.Nq, self.Nfq
        u = ut[:, ks]                                   # (3, k, Nh)
        # physical hybridized operators Q_h^{x,k}, Q_h^{y,k} (Sec. 2.7)
        def phys(Gr, Gs):
            return 0.5 * (ref.Qhr[None] * (Gr[:, :, None] + Gr[:, None, :])
                          + ref.Qhs[None] * (Gs[:, :, None] + Gs[:, None, :]))
        Qx = phys(m.rxJ[ks], m.sxJ[ks])                 # (k, Nh, Nh)
        Qy = phys(m.ryJ[ks], m.syJ[ks])
        # flux matrices (F^i)_{lm} = f_S^i(u~_l, u~_m) (eq. (flux_matrix))
        Fx, Fy = swe.ec_flux(u[:, :, :, None], u[:, :, None, :], g)   # (3, k, Nh, Nh)
        vol_nodes = 2.0 * np.einsum("klm,cklm->ckl", Qx, Fx) + 2.0 * np.einsum("klm,cklm->ckl", Qy, Fy)
        # interface terms V_f^T B^{i,k} (f_S^i(u~+, u~) - f^i(u~))
        uf = u[:, :, Nq:]
        flat = ut[:, :, Nq:].reshape(3, -1)
        idx = (ks[:, None] * Nfq + np.arange(Nfq)[None, :]).ravel()
        uP = flat[:, m.mapP[idx]].reshape(3, ks.size, Nfq)
        nxJ, nyJ, sJ = m.nxJ[ks], m.nyJ[ks], m.sJ[ks]
        if m.walls:
            # reflective wall (Sec. 2.9): exterior h+ = h and u_n+ = -u_n, the
            # tangential velocity kept, i.e. the momentum mirrored in the wall
            wall = np.repeat(m.wall[ks], self.N + 1, axis=1)          # (k, Nfq)
            nx, ny = nxJ / sJ, nyJ / sJ
            hun = uf[1] * nx + uf[2] * ny
            mirror = np.stack([uf[0], uf[1] - 2.0 * hun * nx, uf[2] - 2.0 * hun * ny])
            uP = np.where(wall[None], mirror, uP)
        fSx, fSy = swe.ec_flux(uP, uf, g)
        fx, fy = swe.physical_flux(uf, g)
        wf = ref.wf[None, :]
        surf_nodes = wf * (nxJ * (fSx - fx) + nyJ * (fSy - fy))
        if self.lf:
            nx, ny = nxJ / sJ, nyJ / sJ
            lam = np.maximum(swe.wave_speed(uf, nx, ny, g), swe.wave_speed(uP, nx, ny, g))
            surf_nodes = surf_nodes - wf * 0.5 * lam * sJ * (uP - uf)
        src_nodes = self._source_nodes(u, Qx, Qy, self.bh[ks])
        total = (-np.einsum("hn,ckh->ckn", ref.Vh, vol_nodes)
                 - np.einsum("fn,ckf->ckn", ref.Vf, surf_nodes)
                 + np.einsum("hn,ckh->ckn", ref.Vh, src_nodes))
        if self.forcing is not None:
            fq = self.forcing(m.xq[ks], m.yq[ks], t, g)           # (3, k, Nq)
            total = total + np.einsum("qn,kq,ckq->ckn", ref.Vq * ref.w[:, None], m.Jq[ks], fq)
        return np.einsum("knm,ckm->ckn", m.Mh_inv[ks], total)

    def _source_nodes(self, u, Qx, Qy, bh):
        """Bathymetry source at the hybrid nodes,
        [0; -g diag(h~) Q_h^{x,k} b_h; -g diag(h~) Q_h^{y,k} b_h] (Sec. 2.8)."""
        src = np.zeros_like(u)
        src[1] = -self.g * u[0] * np.einsum("klm,km->kl", Qx, bh)
        src[2] = -self.g * u[0] * np.einsum("klm,km->kl", Qy, bh)
        return src

    # -- term magnitudes (for floating-point error bounds in the tests) ---------------
    def rhs_term_magnitude(self, u_h, t=0.0, elems=None):
        """Per entry of du_h/dt (3, K, Np), or of the listed elements only: the
        sum of the absolute values of every term that eq. (dgform) adds up for
        it, i.e. the right-hand side evaluated with each operator entry, flux
        product, source and penalty term replaced by its absolute value (the
        pressure g{h}^2 - 1/2 g{h^2} by its value 1/2 g h_l h_m, a jump by the
        sum of the two sides).  A floating-point evaluation of the same sums
        with unit roundoff eps has an error of at most a modest multiple of
        eps times this quantity, which is what the tests scale their
        element-wise bounds with.  Not part of the scheme."""
        ks = np.arange(self.K) if elems is None else np.asarray(elems, dtype=np.int64)
        if elems is None:
            ut, _ = self.entropy_projection(u_h)
        else:
            nbr = self.mesh.EToE[ks].ravel()
            need = np.unique(np.concatenate([ks, nbr]))
            ut = np.full((3, self.K, self.Nh), np.nan)
            ut[:, need] = self._entropy_projection_subset(u_h, need)
        ref, m, g = self.ref, self.mesh, self.g
        Nq, Nfq = self.Nq, self.Nfq
        u = ut[:, ks]
        def phys(Gr, Gs):
            return 0.5 * (ref.Qhr[None] * (Gr[:, :, None] + Gr[:, None, :])
                          + ref.Qhs[None] * (Gs[:, :, None] + Gs[:, None, :]))
        aQx = np.abs(phys(m.rxJ[ks], m.sxJ[ks]))
        aQy = np.abs(phys(m.ryJ[ks], m.syJ[ks]))

        def flux_abs(uL, uR):
            # |{hu}| , |{hu}{u}| + |p|, |{hu}{v}| and the y counterparts, p = 1/2 g hL hR
            hL, hR = uL[0], uR[0]
            uA = 0.5 * (uL[1] / hL + uR[1] / hR)
            vA = 0.5 * (uL[2] / hL + uR[2] / hR)
            huA = 0.5 * (np.abs(uL[1]) + np.abs(uR[1]))
            hvA = 0.5 * (np.abs(uL[2]) + np.abs(uR[2]))
            p = 0.5 * g * np.abs(hL * hR)
            fx = np.stack([huA, huA * np.abs(uA) + p, huA * np.abs(vA)])
            fy = np.stack([hvA, hvA * np.abs(uA), hvA * np.abs(vA) + p])
            return fx, fy
        Fx, Fy = flux_abs(u[:, :, :, None], u[:, :, None, :])
        vol = 2.0 * np.einsum("klm,cklm->ckl", aQx, Fx) + 2.0 * np.einsum("klm,cklm->ckl", aQy, Fy)
        uf = u[:, :, Nq:]
        flat = ut[:, :, Nq:].reshape(3, -1)
        idx = (ks[:, None] * Nfq + np.arange(Nfq)[None, :]).ravel()
        uP = flat[:, m.mapP[idx]].reshape(3, ks.size, Nfq)
        nxJ, nyJ, sJ = m.nxJ[ks], m.nyJ[ks], m.sJ[ks]
        if m.walls:
            wall = np.repeat(m.wall[ks], self.N + 1, axis=1)
            nx, ny = nxJ / sJ, nyJ / sJ
            hun = uf[1] * nx + uf[2] * ny
            mirror = np.stack([uf[0], uf[1] - 2.0 * hun * nx, uf[2] - 2.0 * hun * ny])
            uP = np.where(wall[None], mirror, uP)
        fSx, fSy = flux_abs(uP, uf)
        fx, fy = flux_abs(uf, uf)
        wf = ref.wf[None, :]
        surf = wf * (np.abs(nxJ) * (fSx + fx) + np.abs(nyJ) * (fSy + fy))
        if self.lf:
            nx, ny = nxJ / sJ, nyJ / sJ
            lam = np.maximum(swe.wave_speed(uf, nx, ny, g), swe.wave_speed(uP, nx, ny, g))
            surf = surf + wf * 0.5 * lam * sJ * (np.abs(uP) + np.abs(uf))
        src = np.zeros_like(u)
        bh = np.abs(self.bh[ks])
        src[1] = g * np.abs(u[0]) * np.einsum("klm,km->kl", aQx, bh)
        src[2] = g * np.abs(u[0]) * np.einsum("klm,km->kl", aQy, bh)
        aVh, aVf = np.abs(ref.Vh), np.abs(ref.Vf)
        total = (np.einsum("hn,ckh->ckn", aVh, vol) + np.einsum("fn,ckf->ckn", aVf, surf)
                 + np.einsum("hn,ckh->ckn", aVh, src))
        if self.forcing is not None:
            fq = np.abs(self.forcing(m.xq[ks], m.yq[ks], t, g))
            total = total + np.einsum("qn,kq,ckq->ckn", np.abs(ref.Vq) * ref.w[:, None], m.Jq[ks], fq)
        if m.mass == "exact":
            aMinv = np.abs(m.Mh_inv[ks])
        else:
            # the weight-adjusted inverse by its definition M^-1 (Vq^T W diag(1/J) Vq) M^-1
            VqW = ref.Vq * ref.w[:, None]
            Mri = np.abs(np.linalg.inv(VqW.T @ ref.Vq))
            inner = np.einsum("qn,kq,qm->knm", np.abs(VqW), 1.0 / m.Jq[ks], np.abs(ref.Vq))
            aMinv = Mri[None] @ inner @ Mri[None]
        return np.einsum("knm,ckm->ckn", aMinv, total)

    # -- time stepping (Sec. 4) -----------------------------------------------------
    def step(self, u_h, res, t, dt):
        """One LSRK45 step; returns (u_h, res, t + dt)."""
        u_h = u_h.copy()
        res = res.copy()
        for s in range(5):
            r = self.rhs(u_h, t + LSRK45_C[s] * dt)
            res = LSRK45_A[s] * res + dt * r
            u_h = u_h + LSRK45_B[s] * res
        return u_h, res, t + dt

    def run(self, u_h, nsteps, dt=None, t=0.0):
        dt = self.dt() if dt is None else dt
        res = np.zeros_like(u_h)
        for _ in range(nsteps):
            u_h, res, t = self.step(u_h, res, t, dt)
        return u_h, t

    # -- diagnostics -----------------------------------------------------------------
    def entropy(self, u_h):
        """sum_k sum_q w_q J_q S(u_q) (Sec. 2.4)."""
        ref, m = self.ref, self.mesh
        uq = np.einsum("qn,ckn->ckq", ref.Vq, u_h)
        return float(np.sum(ref.w[None, :] * m.Jq * swe.entropy(uq, self.bq, self.g)))

    def mass(self, u_h):
        ref, m = self.ref, self.mesh
        hq = u_h[0] @ ref.Vq.T
        return float(np.sum(ref.w[None, :] * m.Jq * hq))

    def entropy_rate_terms(self, u_h, dudt):
        """Per-element d/dt of the entropy integral, sum_q w_q J_q v(u_q) . (Vq du/dt)_q."""
        ref, m = self.ref, self.mesh
        uq = np.einsum("qn,ckn->ckq", ref.Vq, u_h)
        vq = swe.entropy_vars(uq, self.bq, self.g)
        dq = np.einsum("qn,ckn->ckq", ref.Vq, dudt)
        return np.sum(ref.w[None, :] * m.Jq * np.sum(vq * dq, axis=0), axis=1)

    def l2_error_volq(self, u_h, exact_volq):
        """Per-field L2 error against values (3, K, Nq) given at the volume
        quadrature points, measured with the volume rule itself:
        sqrt(sum_k sum_q w_q J_q (V_q u_h - exact)^2) (the error measure of
        Sec. 4.1 on the element's own rule)."""
        ref, m = self.ref, self.mesh
        e = np.einsum("qn,ckn->ckq", ref.Vq, u_h) - np.asarray(exact_volq, np.float64)
        return np.sqrt(np.sum(ref.w[None, None, :] * m.Jq[None] * e * e, axis=(1, 2)))

    def l2_error(self, u_h, exact):
        """L2 error against exact(x, y) -> (3, K, npts) with the degree >= 2N+2
        rule (Sec. 4.1); returns per-field errors."""
        ref, m = self.ref, self.mesh
        x, y = self.points("errq")
        Vr, Vs = _basis_derivs(ref.N, ref.rq2, ref.sq2)
        xr = m.xmodal @ Vr.T
        xs = m.xmodal @ Vs.T
        yr = m.ymodal @ Vr.T
        ys = m.ymodal @ Vs.T
        J = xr * ys - xs * yr
        uq = np.einsum("qn,ckn->ckq", ref.Vq2, u_h)
        e = uq - exact(x, y)
        return np.sqrt(np.sum(ref.wq2[None, None, :] * J[None] * e * e, axis=(1, 2)))


def _basis_derivs(N, r, s):
    from .refelem import basis
    _, Vr, Vs = basis(N, r, s, derivs=True)
    return Vr, Vs


def default_oracle(**kw):
    return Oracle(**kw)


__all__ = ["Oracle", "Mesh", "RefElem", "LSRK45_A", "LSRK45_B", "LSRK45_C", "mms_sine_forcing"]
