"""Volume terms of the entropy-stable and the traditional DG kernels with
dense operators, for the cost comparison of Sec. 5.4 (oracle; test
infrastructure only).

The comparison replaces the SBP differentiation matrices by square matrices
with random entries and times, per element with n nodes and state u = (h, hu,
hv) at the nodes:

  * traditional DG: the matrix-vector products  r = Q^x f^x(u) + Q^y f^y(u),
    one flux evaluation per node;
  * entropy-stable DG: flux differencing  r = (Q^x o F^x) 1 + (Q^y o F^y) 1,
    F^i_jk = f_S^i(u_j, u_k), one two-point flux evaluation per matrix entry.

Both are written here from their definitions with the fluxes of swe.py
(eq. (SWE) and eqs. (SWE_flux1/2)).  Arrays: Q^x, Q^y are (n, n) with Q[j, k]
multiplying the flux between nodes j and k into row j; u is (3, K, n).
"""

import numpy as np

from .swe import ec_flux, physical_flux


def volume_dg(Qx, Qy, u, g):
    """Traditional DG volume term Q^x f^x + Q^y f^y per element (Sec. 5.4)."""
    fx, fy = physical_flux(u, g)                      # (3, K, n) each
    return np.einsum("jk,cek->cej", Qx, fx) + np.einsum("jk,cek->cej", Qy, fy)


def volume_esdg(Qx, Qy, u, g):
    """ESDG flux-differencing volume term (Q^x o F^x) 1 + (Q^y o F^y) 1 per
    element (Sec. 5.4, with the entropy-conservative fluxes of Sec. 2.8)."""
    out = np.zeros_like(u)
    for e in range(u.shape[1]):
        uj = u[:, e, :, None]                          # node j (rows)
        uk = u[:, e, None, :]                          # node k (columns)
        Fx, Fy = ec_flux(uj, uk, g)                    # (3, n, n)
        out[:, e, :] = (Qx[None] * Fx).sum(axis=2) + (Qy[None] * Fy).sum(axis=2)
    return out
