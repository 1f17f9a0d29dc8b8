"""Element-wise error bounds for the FP32 path (test helper).

FP32 right-hand side.  Every step of the FP32 path is a sum of products
evaluated in FP32 (unit roundoff u = 2^-24).  A computed sum of n terms is
within gamma_n ~ n u of the exact one, measured against the sum of its terms'
absolute values (the standard forward bound of a dot product).  Chained:

  * the entropy projection (Sec. 2.6) evaluates V_q u (Np terms), V_q^T W J v
    (Nq), (M_h^k)^{-1} (Np) and V_h (Np) after rounding the FP64 state to
    FP32, plus pointwise maps (v(u), u(v)) of a few operations each, so the
    entropy-projected values carry a relative error of at most about
    (3 Np + Nq + 8) u (the weight-adjusted inverse replaces (M_h^k)^{-1} by
    two sums of Nq terms: (2 Np + 3 Nq + 8) u);
  * the fluxes are products of at most three such values, which at most
    triples a relative error;
  * the flux differencing sums Nh terms per row, the lift Nh and the inverse
    mass Np (weight-adjusted: Nh, Nq and Nq).

With every partial sum bounded by the magnitude of the final terms (the
oracle's rhs_term_magnitude: the right-hand side with each term by its
absolute value), an entry of du/dt is within

  c u mag,  c = 3 (3 Np + Nq + 8) + 2 Nh + Np + 8

of the exact one (first order in u; the +8 covers the FP32 storage of the
metrics, Jacobians, bathymetry and inverse mass).  DG-SBP (Sec. 3) has no
projection: c = 3 * 4 + Nq + 8 (state rounding and the pointwise record,
the Nq-term pair sums, the division by w J).  A defect confined to one
element or one node (a wrong index, a dropped term) moves its entries by a
sizeable fraction of their terms, far above this bound.

FP32 states.  The parity bar on a state after the configured steps is a
relative 1e-5; besides the relative L2 norm it is applied entry by entry
against the largest entry (a max norm), so an error confined to a few
coefficients cannot hide in the norm of the whole state.
"""

import numpy as np

U32 = 2.0 ** -24


def c_modal(Np, Nq, Nfq, wadg=False):
    Nh = Nq + Nfq
    if wadg:
        return 3 * (2 * Np + 3 * Nq + 8) + Nh + 2 * Nq + 8
    return 3 * (3 * Np + Nq + 8) + 2 * Nh + Np + 8


def c_modal_tc(Np, Nq, Nfq):
    """The same bound with the dense contractions (Vq, Vq^T W J, Vh and the
    lift Vh^T) on the tensor cores: each operand is split into TF32 parts
    x = x_hi + x_lo and a product is formed as a_hi b_hi + a_lo b_hi + a_hi b_lo,
    which leaves |a_lo b_lo| and the roundings of the two lo parts, at most
    3 * 2^-22 = 12 u of |a b|; with the tensor core's FP32 accumulation taken
    at 2 u per addition, a contraction of n terms carries (12 + 2 n) u instead
    of n u.  The three projection contractions enter tripled (as the
    projection does above), the lift once."""
    Nh = Nq + Nfq
    return c_modal(Np, Nq, Nfq) + 3 * (36 + 2 * Np + Nq) + 12 + Nh


def c_sbp(Nq):
    return 3 * 4 + Nq + 8


def check_fp32_rhs(got, want, mag, c):
    """Entry by entry: |got - want| <= c u mag.  Returns the largest ratio
    |got - want| / (u mag), for the message."""
    err = np.abs(np.asarray(got) - np.asarray(want))
    ratio = err / (U32 * mag)
    worst = float(np.nanmax(ratio))
    assert np.all(err <= c * U32 * mag), "entry error %.3g u mag at %s (bound %d u mag)" % (
        worst, np.unravel_index(int(np.nanargmax(ratio)), ratio.shape), c)
    print("[fp32 rhs] worst entry error %.3g u mag (bound %d u mag)" % (worst, c))
    return worst


def check_state(got, want, tol):
    """Relative L2 and max-norm (every entry against the largest) within tol."""
    got, want = np.asarray(got), np.asarray(want)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    relmax = np.abs(got - want).max() / np.abs(want).max()
    assert rel < tol and relmax < tol, "state rel L2 %.3g, rel max %.3g (bound %.1g)" % (rel, relmax, tol)
    print("[state] rel L2 %.3g, rel max %.3g (bound %.1g)" % (rel, relmax, tol))
    return rel, relmax
