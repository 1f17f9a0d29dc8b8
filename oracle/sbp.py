"""Traditional entropy-stable DG-SBP scheme of Sec. 3 (oracle; test
infrastructure only).

Nodal unknowns at the Nq points of an SBP quadrature rule (refelem.py,
rule="sbp"), no entropy projection.  The SBP operators come from the
hybridized ones by Theorem 3.1,

  Q_SBP^i = [I; I_f]^T Q_h^i [I; I_f],

and the entropy-conservative DG-SBP form of Sec. 3.2 is written out literally
per element k, with M = W J^k (the diagonal SBP mass matrix on the curved
element, Sec. 2.7) and u_f = I_f u:

  M du/dt = - sum_{i=x,y} (2 Q_SBP^{i,k} o F^i) 1
            - sum_{i=x,y} I_f^T B^{i,k} (f_S^i(u+, u_f) - f^i(u_f))
            + I_f^T W_f (1/2 lambda sJ (u+ - u_f))                 [LF, Sec. 2.8]
            + S + W J f(x, t)                                        [source, forcing]

Readings (the section states the form for the flux terms only):
  * curved elements: Q_SBP^{i,k} from the physical hybridized operator
    Q_h^{i,k} of Sec. 2.7 by the same selection, and M = W J^k;
  * the bathymetry source S = -g [0; diag(h) Q_SBP^{x,k} b; diag(h) Q_SBP^{y,k} b]
    with b the degree-N polynomial of the bathymetry at the SBP nodes (the
    nodal counterpart of the source of Sec. 2.8);
  * Lax-Friedrichs as in the hybridized scheme, on the nodal face values;
  * initial data: nodal values at the SBP points (SURFACE mode: h = H - b).
"""

import numpy as np

from . import swe
from .esdg import LSRK45_A, LSRK45_B, LSRK45_C
from .mesh import Mesh
from .refelem import RefElem


class SBPOracle:
    """FP64 DG-SBP on the structured periodic (optionally curved) mesh.

    State layout: u[field, element, node], fields (h, hu, hv), nodes of the
    SBP rule.
    """

    def __init__(self, N, nx, ny, x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, ax=0.0, ay=0.0, g=1.0, cfl=0.25,
                 lf=True, forcing=None):
        self.ref = RefElem(N, "sbp")
        self.mesh = Mesh(self.ref, nx, ny, x0, x1, y0, y1, ax, ay)
        self.N, self.K = N, self.mesh.K
        self.g, self.cfl, self.lf, self.forcing = g, cfl, lf, forcing
        ref, m = self.ref, self.mesh
        self.Np, self.Nq, self.Nfq = ref.Np, ref.Nq, ref.Nfq
        self.Veq_inv = np.linalg.inv(ref.Veq)
        self.b_modal = np.zeros((self.K, self.Np))
        self.bq = np.zeros((self.K, self.Nq))
        self.M = ref.w[None, :] * m.Jq                 # diagonal mass, (K, Nq)
        # selection [I; I_f] of Theorem 3.1, (Nh, Nq)
        self.S = np.vstack([np.eye(self.Nq), ref.If])

    # -- operators (Theorem 3.1 on the physical operators of Sec. 2.7) ------------
    def sbp_operators(self, ks):
        """Q_SBP^{x,k}, Q_SBP^{y,k} for the elements ks, (k, Nq, Nq) each."""
        ref, m = self.ref, self.mesh

        def phys(Gr, Gs):
            return 0.5 * (ref.Qhr[None] * (Gr[:, :, None] + Gr[:, None, :])
                          + ref.Qhs[None] * (Gs[:, :, None] + Gs[:, None, :]))
        Qhx = phys(m.rxJ[ks], m.sxJ[ks])
        Qhy = phys(m.ryJ[ks], m.syJ[ks])
        S = self.S
        return (np.einsum("ha,khg,gb->kab", S, Qhx, S), np.einsum("ha,khg,gb->kab", S, Qhy, S))

    def reference_sbp_operators(self):
        """Q_SBP^r, Q_SBP^s on the reference element (Theorem 3.1)."""
        S, ref = self.S, self.ref
        return S.T @ ref.Qhr @ S, S.T @ ref.Qhs @ S

    # -- problem data ---------------------------------------------------------------
    def points(self, kind):
        m = self.mesh
        if kind == "nodal":
            return m.xeq, m.yeq
        if kind == "volq":
            return m.xq, m.yq
        if kind == "faceq":
            return m.xf, m.yf
        raise ValueError(kind)

    def set_bathymetry(self, b_nodal):
        """b: the degree-N interpolant of its values at the equispaced nodes
        (C0 across elements), evaluated at the SBP nodes."""
        self.b_modal = np.asarray(b_nodal, np.float64) @ self.Veq_inv.T
        self.bq = self.b_modal @ self.ref.Vq.T

    def init_state(self, q_nodes, surface=False):
        u = np.array(q_nodes, np.float64)
        if surface:
            u[0] = u[0] - self.bq
        return u

    def dt(self):
        CN = (self.N + 1) * (self.N + 2) / 2.0
        return self.cfl * self.mesh.dx / CN

    # -- right-hand side ------------------------------------------------------------
    def rhs(self, u, t=0.0, chunk=1024):
        out = np.zeros_like(u)
        for k0 in range(0, self.K, chunk):
            ks = np.arange(k0, min(self.K, k0 + chunk))
            out[:, ks] = self._rhs_rows(u, ks, t)
        return out

    def rhs_elements(self, u, elems, t=0.0):
        """du/dt on the listed elements only (no projection couples them: each
        needs its own and its face neighbours' nodal values)."""
        return self._rhs_rows(u, np.asarray(elems, dtype=np.int64), t)

    def _rhs_rows(self, u_all, ks, t):
        ref, m, g = self.ref, self.mesh, self.g
        Nfq = self.Nfq
        u = u_all[:, ks]                                         # (3, k, Nq)
        Qx, Qy = self.sbp_operators(ks)
        Fx, Fy = swe.ec_flux(u[:, :, :, None], u[:, :, None, :], g)   # (3, k, Nq, Nq)
        vol = 2.0 * np.einsum("klm,cklm->ckl", Qx, Fx) + 2.0 * np.einsum("klm,cklm->ckl", Qy, Fy)
        # interface: the face values are the nodal values I_f u
        uf = u[:, :, ref.fmap]                                   # (3, k, Nfq)
        flat = u_all[:, :, ref.fmap].reshape(3, -1)
        idx = (ks[:, None] * Nfq + np.arange(Nfq)[None, :]).ravel()
        uP = flat[:, m.mapP[idx]].reshape(3, ks.size, Nfq)
        nxJ, nyJ, sJ = m.nxJ[ks], m.nyJ[ks], m.sJ[ks]
        fSx, fSy = swe.ec_flux(uP, uf, g)
        fx, fy = swe.physical_flux(uf, g)
        wf = ref.wf[None, :]
        surf = wf * (nxJ * (fSx - fx) + nyJ * (fSy - fy))
        if self.lf:
            nx, ny = nxJ / sJ, nyJ / sJ
            lam = np.maximum(swe.wave_speed(uf, nx, ny, g), swe.wave_speed(uP, nx, ny, g))
            surf = surf - wf * 0.5 * lam * sJ * (uP - uf)
        surf_nodes = np.einsum("fq,ckf->ckq", ref.If, surf)      # I_f^T
        src = np.zeros_like(u)
        b = self.bq[ks]
        src[1] = -g * u[0] * np.einsum("klm,km->kl", Qx, b)
        src[2] = -g * u[0] * np.einsum("klm,km->kl", Qy, b)
        total = -vol - surf_nodes + src
        if self.forcing is not None:
            total = total + self.M[ks][None] * self.forcing(m.xq[ks], m.yq[ks], t, g)
        return total / self.M[ks][None]

    def rhs_term_magnitude(self, u, t=0.0, elems=None):
        """Per entry of du/dt, or of the listed elements only: the sum of the
        absolute values of every term the DG-SBP form adds up for it (each
        operator entry, flux product, source and penalty term by its absolute
        value; the pressure by 1/2 g h_l h_m, a jump by the sum of the two
        sides), divided by the diagonal mass.  The scale of a floating-point
        error bound for the same sums; not part of the scheme."""
        ks = np.arange(self.K) if elems is None else np.asarray(elems, dtype=np.int64)
        ref, m, g = self.ref, self.mesh, self.g
        Nfq = self.Nfq
        uk = u[:, ks]
        Qx, Qy = self.sbp_operators(ks)
        aQx, aQy = np.abs(Qx), np.abs(Qy)

        def flux_abs(uL, uR):
            hL, hR = uL[0], uR[0]
            uA = 0.5 * (uL[1] / hL + uR[1] / hR)
            vA = 0.5 * (uL[2] / hL + uR[2] / hR)
            huA = 0.5 * (np.abs(uL[1]) + np.abs(uR[1]))
            hvA = 0.5 * (np.abs(uL[2]) + np.abs(uR[2]))
            p = 0.5 * g * np.abs(hL * hR)
            fx = np.stack([huA, huA * np.abs(uA) + p, huA * np.abs(vA)])
            fy = np.stack([hvA, hvA * np.abs(uA), hvA * np.abs(vA) + p])
            return fx, fy
        Fx, Fy = flux_abs(uk[:, :, :, None], uk[:, :, None, :])
        vol = 2.0 * np.einsum("klm,cklm->ckl", aQx, Fx) + 2.0 * np.einsum("klm,cklm->ckl", aQy, Fy)
        uf = uk[:, :, ref.fmap]
        flat = u[:, :, ref.fmap].reshape(3, -1)
        idx = (ks[:, None] * Nfq + np.arange(Nfq)[None, :]).ravel()
        uP = flat[:, m.mapP[idx]].reshape(3, ks.size, Nfq)
        nxJ, nyJ, sJ = m.nxJ[ks], m.nyJ[ks], m.sJ[ks]
        fSx, fSy = flux_abs(uP, uf)
        fx, fy = flux_abs(uf, uf)
        wf = ref.wf[None, :]
        surf = wf * (np.abs(nxJ) * (fSx + fx) + np.abs(nyJ) * (fSy + fy))
        if self.lf:
            nx, ny = nxJ / sJ, nyJ / sJ
            lam = np.maximum(swe.wave_speed(uf, nx, ny, g), swe.wave_speed(uP, nx, ny, g))
            surf = surf + wf * 0.5 * lam * sJ * (np.abs(uP) + np.abs(uf))
        surf_nodes = np.einsum("fq,ckf->ckq", np.abs(ref.If), surf)
        src = np.zeros_like(uk)
        b = np.abs(self.bq[ks])
        src[1] = g * np.abs(uk[0]) * np.einsum("klm,km->kl", aQx, b)
        src[2] = g * np.abs(uk[0]) * np.einsum("klm,km->kl", aQy, b)
        total = vol + surf_nodes + src
        if self.forcing is not None:
            total = total + self.M[ks][None] * np.abs(self.forcing(m.xq[ks], m.yq[ks], t, g))
        return total / self.M[ks][None]

    # -- time stepping and diagnostics -------------------------------------------------
    def step(self, u, res, t, dt):
        u = u.copy()
        res = res.copy()
        for s in range(5):
            r = self.rhs(u, t + LSRK45_C[s] * dt)
            res = LSRK45_A[s] * res + dt * r
            u = u + LSRK45_B[s] * res
        return u, res, t + dt

    def run(self, u, nsteps, dt=None, t=0.0):
        dt = self.dt() if dt is None else dt
        res = np.zeros_like(u)
        for _ in range(nsteps):
            u, res, t = self.step(u, res, t, dt)
        return u, t

    def entropy(self, u):
        """sum_k sum_q w_q J_q S(u_q) (Sec. 2.4) on the SBP nodes."""
        return float(np.sum(self.M * swe.entropy(u, self.bq, self.g)))

    def mass(self, u):
        return float(np.sum(self.M * u[0]))

    def entropy_rate_terms(self, u, dudt):
        """Per-element sum_q w_q J_q v(u_q) . du_q/dt."""
        v = swe.entropy_vars(u, self.bq, self.g)
        return np.sum(self.M * np.sum(v * dudt, axis=0), axis=1)

    def l2_error_volq(self, u, exact_volq):
        """Per-field L2 error against values (3, K, Nq) given at the SBP nodes,
        measured with the SBP rule: sqrt(sum_k sum_q w_q J_q (u_q - exact)^2)."""
        e = u - np.asarray(exact_volq, np.float64)
        return np.sqrt(np.sum(self.M[None] * e * e, axis=(1, 2)))

    def l2_error(self, u, exact):
        """Per-field L2 error of the nodal solution, measured with the SBP
        rule itself (the nodal values are the unknowns; Sec. 3)."""
        x, y = self.points("volq")
        e = u - exact(x, y)
        return np.sqrt(np.sum(self.M[None] * e * e, axis=(1, 2)))
