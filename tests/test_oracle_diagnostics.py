"""Pins of the oracle's diagnostics: the total entropy and mass integrals of
Sec. 2.4 (the entropy S(u) = 1/2 h (u^2 + v^2) + 1/2 g h^2 + g h b, whose
integral Theorem 2.2 bounds) and the per-element entropy rate, for the modal
ESDG oracle and the DG-SBP oracle of Sec. 3.

Each check compares the oracle with something other than its own
quadrature: a closed form for a constant state on a curved periodic mesh
(the curving keeps the area of [-1,1]^2), an exact symbolic integral of
polynomial data on an affine mesh, and the derivative of the (pinned)
entropy integral along a direction.  The last group plants plausible
mistakes in the oracle's diagnostics (a dropped Jacobian, a dropped
bathymetry term, equal weights in place of the rule's) and shows that a pin
fails for each.
"""

import numpy as np
import pytest

from oracle import Oracle
from oracle.sbp import SBPOracle
from oracle import swe

sp = pytest.importorskip("sympy")

G = 1.3                            # a gravity other than 1, so a dropped g shows
H0, U0, V0, B0 = 1.7, 0.3, -0.2, 0.25


def _const_closed_form(area):
    S = 0.5 * H0 * (U0 * U0 + V0 * V0) + 0.5 * G * H0 * H0 + G * H0 * B0
    return area * S, area * H0


def _const_state(o, modal):
    K = o.K
    o.set_bathymetry(np.full((K, o.Np), B0))
    n = o.Nq
    q = np.stack([np.full((K, n), H0), np.full((K, n), H0 * U0), np.full((K, n), H0 * V0)])
    return o.init_state(q)


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_modal_entropy_and_mass_of_a_constant_state_on_a_curved_mesh(N, rule):
    """A constant state over a constant bottom: S_tot = 4 S(h0, u0, v0; b0) and
    mass = 4 h0, since the curved periodic mesh of [-1,1]^2 keeps its area
    (its warp vanishes on the boundary) and the volume rule integrates the
    degree-2N-2 Jacobian exactly."""
    o = Oracle(N, 5, 4, ax=0.05, ay=0.05, g=G, rule=rule)
    u = _const_state(o, True)
    S_ex, M_ex = _const_closed_form(4.0)
    assert abs(o.entropy(u) - S_ex) <= 1e-13 * S_ex
    assert abs(o.mass(u) - M_ex) <= 1e-13 * M_ex


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sbp_entropy_and_mass_of_a_constant_state_on_a_curved_mesh(N):
    o = SBPOracle(N, 5, 4, ax=0.05, ay=0.05, g=G)
    u = _const_state(o, False)
    S_ex, M_ex = _const_closed_form(4.0)
    assert abs(o.entropy(u) - S_ex) <= 1e-13 * S_ex
    assert abs(o.mass(u) - M_ex) <= 1e-13 * M_ex


# A rectangle other than [-1,1]^2 (area 4.5), so that no hard-coded area passes.
X0, X1, Y0, Y1 = 0.0, 3.0, -1.0, 0.5


def _poly_data(deg_h, deg_b, seed):
    """Random polynomials h (positive on the rectangle) and b in x, y, as sympy
    expressions and numpy callables."""
    x, y = sp.symbols("x y")
    rng = np.random.default_rng(seed)

    def poly(deg, scale):
        return sum(sp.Rational(int(rng.integers(-9, 10)), 10) * scale * x ** i * y ** j
                   for i in range(deg + 1) for j in range(deg + 1 - i))
    # shift the argument to the rectangle's centre so h stays near 3
    xs, ys = x - 1.5, y + 0.25
    h = 3 + poly(deg_h, sp.Rational(1, 10)).subs({x: xs, y: ys}, simultaneous=True)
    b = poly(deg_b, sp.Rational(1, 10)).subs({x: xs, y: ys}, simultaneous=True)
    return x, y, sp.expand(h), sp.expand(b)


def _exact_integrals(x, y, h, b):
    S = sp.Rational(1, 2) * h * (sp.nsimplify(U0) ** 2 + sp.nsimplify(V0) ** 2) \
        + sp.Rational(1, 2) * sp.nsimplify(G) * h ** 2 + sp.nsimplify(G) * h * b
    S_int = sp.integrate(sp.integrate(sp.expand(S), (x, X0, X1)), (y, Y0, Y1))
    M_int = sp.integrate(sp.integrate(h, (x, X0, X1)), (y, Y0, Y1))
    return float(S_int), float(M_int)


def _fill(o, x, y, h, b, modal):
    fh = sp.lambdify((x, y), h, "numpy")
    fb = sp.lambdify((x, y), b, "numpy")
    xb, yb = o.points("nodal")
    o.set_bathymetry(np.broadcast_to(fb(xb, yb), xb.shape).astype(np.float64))
    xq, yq = o.points("volq")
    hq = np.broadcast_to(fh(xq, yq), xq.shape).astype(np.float64)
    return o.init_state(np.stack([hq, U0 * hq, V0 * hq]))


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("N", [1, 2, 3])
def test_modal_entropy_and_mass_of_polynomial_data_on_an_affine_mesh(N, rule):
    """h, b of degree N and a constant velocity on affine elements: the
    projection reproduces them, S(u) is a polynomial of degree 2N, which the
    volume rule integrates exactly, so the oracle's integrals equal the exact
    symbolic ones.  A transposed operator, a wrong weight or Jacobian, or a
    term of S with a wrong factor does not."""
    x, y, h, b = _poly_data(N, N, seed=10 + N)
    o = Oracle(N, 4, 3, X0, X1, Y0, Y1, g=G, rule=rule)
    u = _fill(o, x, y, h, b, True)
    S_ex, M_ex = _exact_integrals(x, y, h, b)
    assert abs(o.entropy(u) - S_ex) <= 1e-12 * abs(S_ex)
    assert abs(o.mass(u) - M_ex) <= 1e-12 * abs(M_ex)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sbp_entropy_and_mass_of_polynomial_data_on_an_affine_mesh(N):
    """The SBP rules are exact to degree 2N - 1: with h of degree N - 1 and b
    of degree N, every term of S(u) (degrees N - 1, 2N - 2, 2N - 1) is
    integrated exactly by the nodal sums."""
    x, y, h, b = _poly_data(N - 1, N, seed=20 + N)
    o = SBPOracle(N, 4, 3, X0, X1, Y0, Y1, g=G)
    u = _fill(o, x, y, h, b, False)
    S_ex, M_ex = _exact_integrals(x, y, h, b)
    assert abs(o.entropy(u) - S_ex) <= 1e-12 * abs(S_ex)
    assert abs(o.mass(u) - M_ex) <= 1e-12 * abs(M_ex)


def _random_modal(o, seed):
    rng = np.random.default_rng(seed)
    u = 0.05 * rng.standard_normal((3, o.K, o.Np))
    u[0, :, 0] += 2.0
    return u


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
def test_modal_entropy_rate_terms_are_the_derivative_of_the_entropy(rule):
    """sum_k of the per-element rate terms for a direction d equals
    d/de S_tot(u + e d) at e = 0 (a central difference of the pinned entropy
    integral): the rate is v(u_q) . (V_q d)_q integrated with w J."""
    o = Oracle(3, 4, 4, ax=0.05, ay=0.05, g=G, rule=rule)
    xb, yb = o.points("nodal")
    o.set_bathymetry(0.1 * np.sin(np.pi * xb) * np.cos(np.pi * yb))
    u = _random_modal(o, 1)
    d = np.random.default_rng(2).standard_normal(u.shape)
    eps = 1e-5
    fd = (o.entropy(u + eps * d) - o.entropy(u - eps * d)) / (2 * eps)
    rate = o.entropy_rate_terms(u, d).sum()
    assert abs(rate - fd) <= 1e-8 * abs(fd)


def test_sbp_entropy_rate_terms_are_the_derivative_of_the_entropy():
    o = SBPOracle(3, 4, 4, ax=0.05, ay=0.05, g=G)
    xb, yb = o.points("nodal")
    o.set_bathymetry(0.1 * np.sin(np.pi * xb) * np.cos(np.pi * yb))
    rng = np.random.default_rng(3)
    u = 0.05 * rng.standard_normal((3, o.K, o.Nq))
    u[0] += 2.0
    d = rng.standard_normal(u.shape)
    eps = 1e-5
    fd = (o.entropy(u + eps * d) - o.entropy(u - eps * d)) / (2 * eps)
    rate = o.entropy_rate_terms(u, d).sum()
    assert abs(rate - fd) <= 1e-8 * abs(fd)


# ---------------------------------------------------------------------------
# Planted mistakes in the diagnostics: each must fail one of the pins above
# ---------------------------------------------------------------------------


def _entropy_without_J(o):
    def f(u_h):
        uq = np.einsum("qn,ckn->ckq", o.ref.Vq, u_h)
        return float(np.sum(o.ref.w[None, :] * swe.entropy(uq, o.bq, o.g)))
    return f


def _mass_without_J(o):
    def f(u_h):
        return float(np.sum(o.ref.w[None, :] * (u_h[0] @ o.ref.Vq.T)))
    return f


def _entropy_without_b(o):
    def f(u_h):
        uq = np.einsum("qn,ckn->ckq", o.ref.Vq, u_h)
        return float(np.sum(o.ref.w[None, :] * o.mesh.Jq * swe.entropy(uq, 0.0 * o.bq, o.g)))
    return f


def test_planted_dropped_jacobian_fails_the_constant_state_pin(monkeypatch):
    o = Oracle(3, 5, 4, ax=0.05, ay=0.05, g=G)
    u = _const_state(o, True)
    S_ex, M_ex = _const_closed_form(4.0)
    assert abs(o.entropy(u) - S_ex) <= 1e-13 * S_ex
    monkeypatch.setattr(o, "entropy", _entropy_without_J(o))
    monkeypatch.setattr(o, "mass", _mass_without_J(o))
    assert abs(o.entropy(u) - S_ex) > 1e-3 * S_ex
    assert abs(o.mass(u) - M_ex) > 1e-3 * M_ex


def test_planted_dropped_bathymetry_term_fails_the_constant_state_pin(monkeypatch):
    o = Oracle(2, 5, 4, ax=0.05, ay=0.05, g=G)
    u = _const_state(o, True)
    S_ex, _ = _const_closed_form(4.0)
    monkeypatch.setattr(o, "entropy", _entropy_without_b(o))
    assert abs(o.entropy(u) - S_ex) > 1e-3 * S_ex


def test_planted_equal_weights_fail_the_polynomial_pin(monkeypatch):
    """Equal weights 2 / Nq still integrate constants (they sum to the
    reference area), so only the polynomial pin catches them."""
    N = 3
    x, y, h, b = _poly_data(N, N, seed=10 + N)
    o = Oracle(N, 4, 3, X0, X1, Y0, Y1, g=G)
    u = _fill(o, x, y, h, b, True)
    S_ex, M_ex = _exact_integrals(x, y, h, b)
    w_equal = np.full_like(o.ref.w, o.ref.w.sum() / o.ref.w.size)
    monkeypatch.setattr(o.ref, "w", w_equal)
    assert abs(o.entropy(u) - S_ex) > 1e-6 * abs(S_ex)
    assert abs(o.mass(u) - M_ex) > 1e-6 * abs(M_ex)


def test_planted_dropped_jacobian_fails_the_sbp_constant_state_pin(monkeypatch):
    o = SBPOracle(3, 5, 4, ax=0.05, ay=0.05, g=G)
    u = _const_state(o, False)
    S_ex, M_ex = _const_closed_form(4.0)
    monkeypatch.setattr(o, "M", np.broadcast_to(o.ref.w[None, :], o.M.shape))
    assert abs(o.entropy(u) - S_ex) > 1e-3 * S_ex
    assert abs(o.mass(u) - M_ex) > 1e-3 * M_ex


# ---------------------------------------------------------------------------
# The term magnitude used to scale the FP32 error bounds of the GPU tests
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("mass", ["exact", "weight_adjusted"])
def test_modal_term_magnitude_bounds_the_right_hand_side(mass, walls):
    """By the triangle inequality the sum of the absolute values of the terms
    bounds the sum itself, entry by entry; on listed elements it equals the
    whole-mesh value; and with u = v = 0, b = 0 and no LF every term is a
    pressure term, quadratic in h (so doubling h multiplies it by 4)."""
    from oracle.esdg import mms_sine_forcing
    o = Oracle(3, 5, 4, ax=0.05, ay=0.05, g=G, rule="symmetric", mass=mass, walls=walls,
               forcing=mms_sine_forcing)
    xb, yb = o.points("nodal")
    o.set_bathymetry(0.1 * np.sin(np.pi * xb) * np.cos(np.pi * yb))
    u = _random_modal(o, 4)
    r = o.rhs(u, 0.3)
    m = o.rhs_term_magnitude(u, 0.3)
    assert np.all(np.abs(r) <= m * (1 + 1e-12))
    ks = [0, 3, o.K - 1]
    assert np.allclose(o.rhs_term_magnitude(u, 0.3, elems=ks), m[:, ks], rtol=1e-14, atol=0)
    o2 = Oracle(3, 5, 4, ax=0.05, ay=0.05, g=G, rule="symmetric", mass=mass, walls=walls, lf=False)
    h = np.zeros_like(u)
    h[0, :, 0] = 1.5 * np.sqrt(2.0)        # a constant depth (the mode-0 value is sqrt(2) h)
    m1, m2 = o2.rhs_term_magnitude(h), o2.rhs_term_magnitude(2.0 * h)
    assert np.allclose(m2, 4.0 * m1, rtol=1e-13, atol=0)


def test_sbp_term_magnitude_bounds_the_right_hand_side():
    o = SBPOracle(3, 5, 4, ax=0.05, ay=0.05, g=G)
    xb, yb = o.points("nodal")
    o.set_bathymetry(0.1 * np.sin(np.pi * xb) * np.cos(np.pi * yb))
    rng = np.random.default_rng(6)
    u = 0.05 * rng.standard_normal((3, o.K, o.Nq))
    u[0] += 2.0
    r = o.rhs(u)
    m = o.rhs_term_magnitude(u)
    assert np.all(np.abs(r) <= m * (1 + 1e-12))
    ks = [1, 2, o.K - 1]
    assert np.allclose(o.rhs_term_magnitude(u, elems=ks), m[:, ks], rtol=1e-14, atol=0)
