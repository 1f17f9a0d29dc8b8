"""Pins of the DG-SBP oracle (Sec. 3; oracle/sbp.py, the SBP rules of
oracle/refelem.py): the rule against exact integrals and the stated
properties, the operators against Theorem 3.1's SBP property and exactness,
and the scheme against the invariants of Theorem 2.2 and the manufactured
solution.  CPU only."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.esdg import mms_sine_forcing
from oracle.refelem import face_quadrature, sbp_quadrature
from oracle.sbp import SBPOracle


def _monomial_integral(a, b):
    """int over the reference triangle of r^a s^b (Dirichlet integral, exact
    rational arithmetic)."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            c = math.comb(a, i) * math.comb(b, j) * 2 ** (i + j) * (-1) ** (a - i + b - j)
            tot += Fraction(c * math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
    return float(4 * tot)


def _bary(r, s):
    return np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=1)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_sbp_rule_properties(N):
    """Sec. 3.1: positive weights, exact to degree 2N-1, the N+1
    Gauss-Legendre points of every face among the nodes; here also fully
    symmetric with the remaining nodes strictly inside."""
    r, s, w = sbp_quadrature(N)
    assert np.all(w > 0)
    d = 2 * N - 1
    for a in range(d + 1):
        for b in range(d + 1 - a):
            exact = _monomial_integral(a, b)
            assert abs(np.sum(w * r ** a * s ** b) - exact) < 1e-13, (a, b)
    rf, sf, _, _, _ = face_quadrature(N)
    dist = np.hypot(rf[:, None] - r[None], sf[:, None] - s[None]).min(axis=1)
    assert dist.max() < 1e-13
    on_edge = (np.abs(s + 1) < 1e-12) | (np.abs(r + 1) < 1e-12) | (np.abs(r + s) < 1e-12)
    assert on_edge.sum() == 3 * (N + 1)
    assert np.all(r[~on_edge] > -1) and np.all(s[~on_edge] > -1) and np.all(r[~on_edge] + s[~on_edge] < 0)
    lam = _bary(r, s)
    key = {tuple(np.round(np.r_[lam[i], w[i]], 10)) for i in range(r.size)}
    for perm in [(1, 2, 0), (1, 0, 2)]:     # generators of the triangle's symmetry group
        keyp = {tuple(np.round(np.r_[lam[i][list(perm)], w[i]], 10)) for i in range(r.size)}
        assert keyp == key


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sbp_operators_theorem_3_1(N):
    """Q_SBP = [I; I_f]^T Q_h [I; I_f] is an SBP operator: Q + Q^T = I_f^T B I_f,
    D = M_SBP^{-1} Q differentiates P^N exactly, Q 1 = 0."""
    o = SBPOracle(N, 3, 3)
    ref = o.ref
    Qr, Qs = o.reference_sbp_operators()
    Br = ref.If.T @ np.diag(ref.wf * ref.nr) @ ref.If
    Bs = ref.If.T @ np.diag(ref.wf * ref.ns) @ ref.If
    assert np.abs(Qr + Qr.T - Br).max() < 1e-13 and np.abs(Qs + Qs.T - Bs).max() < 1e-13
    assert np.abs(Qr.sum(1)).max() < 1e-13 and np.abs(Qs.sum(1)).max() < 1e-13
    Dr, Ds = Qr / ref.w[:, None], Qs / ref.w[:, None]
    r, s = ref.rq, ref.sq
    for i in range(N + 1):
        for j in range(N + 1 - i):
            p = r ** i * s ** j
            pr = i * r ** max(i - 1, 0) * s ** j
            ps = j * r ** i * s ** max(j - 1, 0)
            assert np.abs(Dr @ p - pr).max() < 1e-12 and np.abs(Ds @ p - ps).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3])
def test_sbp_physical_operators_on_curved_elements(N):
    """On curved elements Q_SBP^{x,k} + (Q_SBP^{x,k})^T = I_f^T W_f diag(nxJ) I_f
    (and y), and Q_SBP^{i,k} 1 = 0 (the discrete metric identities)."""
    o = SBPOracle(N, 4, 4, ax=0.05, ay=0.05)
    ks = np.arange(o.K)
    Qx, Qy = o.sbp_operators(ks)
    If, wf = o.ref.If, o.ref.wf
    for Q, nJ in ((Qx, o.mesh.nxJ), (Qy, o.mesh.nyJ)):
        B = np.einsum("fa,kf,fb->kab", If, wf[None] * nJ, If)
        assert np.abs(Q + Q.transpose(0, 2, 1) - B).max() < 1e-13
        assert np.abs(Q.sum(2)).max() < 1e-13


def _smooth(o, seed=0, amp=0.01):
    x, y = o.points("volq")
    q = np.stack([2 + 0.1 * np.sin(np.pi * x) * np.cos(np.pi * y) + 0.05 * np.cos(2 * np.pi * y),
                  0.3 * np.cos(np.pi * y), 0.2 * np.sin(np.pi * x)])
    return q + amp * np.random.default_rng(seed).standard_normal(q.shape)


def _bathy(o, amp=0.2):
    xb, yb = o.points("nodal")
    o.set_bathymetry(amp * np.sin(np.pi * xb) * np.sin(np.pi * yb))


@pytest.mark.parametrize("warp", [0.0, 0.05])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sbp_entropy_conservation_mass_and_lf(N, warp):
    """The DG-SBP form is entropy conservative with the EC flux (rate zero),
    conserves mass, and Lax-Friedrichs makes the rate negative."""
    o = SBPOracle(N, 4, 4, ax=warp, ay=warp, lf=False)
    _bathy(o)
    u = _smooth(o)
    r = o.rhs(u)
    terms = o.entropy_rate_terms(u, r)
    assert abs(terms.sum()) < 1e-13 * np.abs(terms).sum()
    assert abs(np.sum(o.M * r[0])) < 1e-13
    o.lf = True
    assert o.entropy_rate_terms(u, o.rhs(u)).sum() < 0


@pytest.mark.parametrize("warp", [0.0, 0.05])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_sbp_lake_at_rest_and_free_stream(N, warp):
    o = SBPOracle(N, 4, 4, ax=warp, ay=warp)
    _bathy(o)
    x, y = o.points("volq")
    u = o.init_state(np.stack([2.0 + 0 * x, 0 * x, 0 * x]), surface=True)
    assert np.abs(o.rhs(u)).max() < 1e-12
    o2 = SBPOracle(N, 4, 4, ax=warp, ay=warp)
    assert np.abs(o2.rhs(np.stack([2.0 + 0 * x, 0.3 + 0 * x, -0.2 + 0 * x]))).max() < 1e-12


def _mms_exact(x, y, t):
    h = 2.0 + 0.1 * np.sin(np.pi * (x + y - t))
    return np.stack([h, 0.5 * h, 0.5 * h])


def _mms_dt_exact(x, y, t):
    ht = -0.1 * np.pi * np.cos(np.pi * (x + y - t))
    return np.stack([ht, 0.5 * ht, 0.5 * ht])


def _mms_oracle(N, nx):
    o = SBPOracle(N, nx, nx, ax=0.05, ay=0.05, forcing=mms_sine_forcing)
    xb, yb = o.points("nodal")
    o.set_bathymetry(0.1 * np.cos(np.pi * xb) * np.cos(np.pi * yb))
    return o


def _consistency(o, t=0.3):
    x, y = o.points("volq")
    r = o.rhs(_mms_exact(x, y, t), t)
    return np.sqrt(np.sum(o.M[None] * (r - _mms_dt_exact(x, y, t)) ** 2))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_sbp_l2_error_volq_closed_form_on_curved_mesh(N):
    """u = 0 against per-field constants c: the error is c times the square
    root of the area of [-1,1]^2 (the SBP rule, exact to 2N-1, integrates the
    degree-2N-2 Jacobian exactly, and the periodic curving keeps the area)."""
    o = SBPOracle(N, 5, 4, ax=0.05, ay=0.05)
    ex = np.stack([np.full((o.K, o.Nq), c) for c in (1.0, 2.0, 3.0)])
    err = o.l2_error_volq(np.zeros((3, o.K, o.Nq)), ex)
    assert np.allclose(err, 2.0 * np.array([1.0, 2.0, 3.0]), rtol=1e-12, atol=0)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_sbp_manufactured_solution_converges(N):
    """Manufactured solution with forcing on curved meshes: the L2 error at
    T = 0.1 falls at least at rate N, and the right-hand side of the exact
    solution approaches its exact time derivative."""
    errs, cons = [], []
    for nx in (4, 8):
        o = _mms_oracle(N, nx)
        x, y = o.points("volq")
        T = 0.1
        n = int(np.ceil(T / o.dt()))
        u, _ = o.run(_mms_exact(x, y, 0.0), n, T / n)
        errs.append(o.l2_error(u, lambda x, y: _mms_exact(x, y, T))[0])
        cons.append(_consistency(o))
    assert np.log2(errs[0] / errs[1]) > N
    assert cons[1] < cons[0] / 2 ** (N - 1)


def test_planted_missing_factor_two_breaks_sbp_consistency(monkeypatch):
    """The DG-SBP form carries 2 Q_SBP o F; with Q_SBP o F instead the right-
    hand side of a smooth exact solution misses its time derivative by O(1)."""
    o = _mms_oracle(3, 8)
    good = _consistency(o)
    real = np.einsum

    def half(spec, *ops, **kw):
        out = real(spec, *ops, **kw)
        return 0.5 * out if spec == "klm,cklm->ckl" else out
    monkeypatch.setattr(np, "einsum", half)
    bad = _consistency(o)
    assert bad > 20 * good
