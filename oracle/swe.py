"""Shallow water physics (oracle; test infrastructure only).

Conservative variables u = (h, hu, hv) with bathymetry b and gravity g.

  * SWE system: eq. (SWE), Sec. 1 (the y-momentum source is read as -g h b_y;
    the printed -g h b_x is a typo).
  * entropy S(u) = 1/2 h (u^2 + v^2) + 1/2 g h^2 + g h b: eq. (entropy_function), Sec. 2.4.
  * entropy variables v = S'(u): Sec. 2.4; the inverse map u(v) is the one
    implied in Sec. 2.6 (u-tilde = u(v-tilde)).
  * entropy-conservative fluxes f_S^x, f_S^y: eqs. (SWE_flux1), (SWE_flux2),
    Sec. 2.8, with {a} = (a_L + a_R)/2 and {h^2} = (h_L^2 + h_R^2)/2.
  * entropy potential psi^i = v^T f^i - F^i; for the SWE with b equal on both
    sides this is psi^x = 1/2 g h^2 u, psi^y = 1/2 g h^2 v (derived from the
    definitions of Sec. 2.4 with the entropy flux F^x = (S + 1/2 g h^2) u ...
    plus the g h b u term, which cancels in v^T f - F).
Arrays carry the field index first: u[0] = h, u[1] = hu, u[2] = hv.
"""

import numpy as np


def physical_flux(u, g):
    """Continuous fluxes f^x(u), f^y(u) of eq. (SWE)."""
    h, hu, hv = u[0], u[1], u[2]
    uu, vv = hu / h, hv / h
    p = 0.5 * g * h * h
    fx = np.stack([hu, hu * uu + p, hu * vv])
    fy = np.stack([hv, hv * uu, hv * vv + p])
    return fx, fy


def entropy(u, b, g):
    """S(u) = 1/2 h (u^2+v^2) + 1/2 g h^2 + g h b (Sec. 2.4)."""
    h, hu, hv = u[0], u[1], u[2]
    return 0.5 * (hu * hu + hv * hv) / h + 0.5 * g * h * h + g * h * b


def entropy_vars(u, b, g):
    """v1 = g(h+b) - 1/2(u^2+v^2), v2 = u, v3 = v (Sec. 2.4)."""
    h, hu, hv = u[0], u[1], u[2]
    uu, vv = hu / h, hv / h
    return np.stack([g * (h + b) - 0.5 * (uu * uu + vv * vv), uu, vv])


def cons_vars(v, b, g):
    """Inverse of entropy_vars: h = (v1 + 1/2(v2^2+v3^2))/g - b, hu = h v2, hv = h v3."""
    h = (v[0] + 0.5 * (v[1] * v[1] + v[2] * v[2])) / g - b
    return np.stack([h, h * v[1], h * v[2]])


def ec_flux(uL, uR, g):
    """Entropy-conservative two-point fluxes (f_S^x, f_S^y), eqs. (SWE_flux1/2)."""
    hL, huL, hvL = uL[0], uL[1], uL[2]
    hR, huR, hvR = uR[0], uR[1], uR[2]
    uLv, vLv = huL / hL, hvL / hL
    uRv, vRv = huR / hR, hvR / hR
    h_avg = 0.5 * (hL + hR)
    h2_avg = 0.5 * (hL * hL + hR * hR)
    hu_avg = 0.5 * (huL + huR)
    hv_avg = 0.5 * (hvL + hvR)
    u_avg = 0.5 * (uLv + uRv)
    v_avg = 0.5 * (vLv + vRv)
    p = g * h_avg * h_avg - 0.5 * g * h2_avg
    fx = np.stack([hu_avg, hu_avg * u_avg + p, hu_avg * v_avg])
    fy = np.stack([hv_avg, hv_avg * u_avg, hv_avg * v_avg + p])
    return fx, fy


def entropy_potential(u, g):
    """psi^x = 1/2 g h^2 u, psi^y = 1/2 g h^2 v (zero bathymetry)."""
    h, hu, hv = u[0], u[1], u[2]
    return 0.5 * g * h * hu, 0.5 * g * h * hv


def wave_speed(u, nx, ny, g):
    """|u.n| + sqrt(g h) for a unit normal (nx, ny): the Lax-Friedrichs
    penalty constant of Sec. 2.8 (the paper does not print it; this is the
    usual local maximum wave speed)."""
    h = u[0]
    un = (u[1] * nx + u[2] * ny) / h
    return np.abs(un) + np.sqrt(g * h)
