"""GPU parity of the weight-adjusted inverse mass (ESDG_MASS_WEIGHT_ADJUSTED,
the alternative to stored inverses that Sec. 2.8 names) against the oracle's
mass="weight_adjusted" on the same seeded inputs.

Tolerances as for the stored inverse: FP64 relative 1e-12 on the right-hand
side and on the state after every step; FP32 right-hand side 5e-5 relative,
FP32 state after the configured steps 1e-5.
"""

import dataclasses

import numpy as np
import pytest

from oracle import Oracle
from oracle.esdg import mms_sine_forcing
from paper_2005_02516_gb300 import workloads as W
from paper_2005_02516_gb300.workloads import random_modal_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WA = "weight_adjusted"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2005_02516_gb300 import esdg
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


def _pair(w, precision, N, nx, ny, rule, lf=True):
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL, Solver
    s = Solver(N, nx, ny, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, lax_friedrichs=lf,
               forcing=w.forcing, rule=rule, mass=WA)
    o = Oracle(N, nx, ny, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, lf=lf,
               forcing=mms_sine_forcing if w.forcing == "mms_sine" else None, rule=rule, mass=WA)
    xb, yb = s.points(ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    return s, o


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


from _bounds import c_modal, check_fp32_rhs, check_state  # noqa: E402


CASES = [
    # (workload, N, nx, ny): curved meshes (MMS carries its forcing term,
    # which the FP32 kernel lifts through A = Vq Vq^T), several tiles and
    # ragged tails; LAKE_BUMP is affine, where the two inverses coincide
    (W.LAKE_BUMP, 2, 8, 8),
    (W.MMS, 3, 5, 4),
    (W.MMS, 4, 3, 5),
    (W.DAM, 4, 6, 5),
    (W.DAM, 5, 4, 3),
    (dataclasses.replace(W.DAM, warp=0.05), 1, 5, 3),
]


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("w,N,nx,ny", CASES)
def test_weight_adjusted_rhs_matches_oracle(w, N, nx, ny, rule):
    for precision, tol in (("fp64", 1e-12), ("fp32", 5e-5)):
        s, o = _pair(w, precision, N, nx, ny, rule)
        u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 40 + N)
        s.set_state(u)
        got = s.rhs(0.23).cpu().numpy()
        want = o.rhs(u, 0.23)
        assert _rel(got, want) < tol, precision
        if precision == "fp32":
            check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.23), c_modal(o.Np, o.Nq, o.Nfq, wadg=True))
        s.close()


@pytest.mark.parametrize("rule,N", [("symmetric", 4), ("collapsed", 3)])
def test_weight_adjusted_steps_match_oracle(rule, N):
    """The manufactured solution (curved 6 x 5 mesh, forcing term): FP64 per
    step at 1e-12 for 15 steps (init_state's host projection included), FP32
    after the same 15 steps at 1e-5."""
    w = dataclasses.replace(W.scaled(W.MMS, 6, 5), N=N, rule=rule)
    s64, o = _pair(w, "fp64", N, 6, 5, rule)
    s32, _ = _pair(w, "fp32", N, 6, 5, rule)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s64.points(ESDG_POINTS_VOLQ)
    s64.init_state(None, w.initial(xs, ys))
    xq, yq = o.points("volq")
    u = o.init_state(w.initial(xq, yq))
    assert _rel(s64.get_state(), u) < 1e-13
    s32.set_state(u)
    res = np.zeros_like(u)
    t, dt = 0.0, o.dt()
    for n in range(15):
        u, res, t = o.step(u, res, t, dt)
        s64.step(1, dt, t - dt)
        assert _rel(s64.get_state(), u) < 1e-12, n
    s32.step(15, dt, 0.0)
    check_state(s32.get_state(), u, 1e-5)


def test_weight_adjusted_entropy_identity_on_gpu():
    """With the EC flux alone the entropy rate that esdg_entropy reports
    vanishes on curved elements: the same weight-adjusted matrix in the
    projection and in the update keeps Theorem 2.2's identity."""
    w = dataclasses.replace(W.LAKE_BUMP, warp=0.05)
    s, o = _pair(w, "fp64", 4, 6, 6, "symmetric", lf=False)
    u = random_modal_state(o.K, o.Np, seed=9)
    s.set_state(u)
    S, M, R = s.entropy(0.0)
    terms = o.entropy_rate_terms(u, o.rhs(u))
    assert abs(R) < 1e-12 * np.abs(terms).sum()
    assert abs(S - o.entropy(u)) < 1e-12 * abs(S)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_weight_adjusted_full_size_sampled_rhs(precision):
    """The smoothed dam break at full size (N=4, K=131072 curved, the 16-point
    symmetric rule) with the weight-adjusted inverse: the right-hand side on
    every 997th element (and the last) against the oracle element by element;
    FP64 at 1e-12, FP32 entry by entry within the first-order FP32 bound
    c u mag (tests/_bounds.py)."""
    w = W.DAM
    s, o = _pair(w, precision, w.N, w.nx, w.nx, w.rule)
    xo, yo = o.points("volq")
    u = o.init_state(w.initial(xo, yo))
    s.set_state(u)
    ks = np.unique(np.concatenate([np.arange(0, o.K, 997), [o.K - 1]]))
    got = s.rhs(0.0).cpu().numpy()[:, ks]
    want = o.rhs_elements(u, ks)
    if precision == "fp64":
        assert _rel(got, want) < 1e-12
    else:
        check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0, elems=ks), c_modal(o.Np, o.Nq, o.Nfq, wadg=True))


def test_weight_adjusted_is_refused_by_ensembles_and_served_fp32():
    from paper_2005_02516_gb300 import esdg
    w = W.LAKE_BUMP
    s = esdg.Solver(2, 8, 8, precision="fp32", warp=0.05, rule="symmetric", mass=WA)
    with pytest.raises(esdg.EsdgError) as ei:
        esdg.Ensemble([s])
    assert ei.value.code == esdg.ESDG_EINVAL
    s.close()
    p = esdg.Problem(2, 8, 8, precision="fp32", warp=0.05, rule="symmetric", mass=WA)
    xb, yb = p.points(esdg.ESDG_POINTS_NODAL)
    xq, yq = p.points(esdg.ESDG_POINTS_VOLQ)
    srv = esdg.Server(hbm_budget_bytes=1 << 30)
    with pytest.raises(esdg.EsdgError) as ei:
        srv.submit(p, w.bathymetry(xb, yb), w.initial(xq, yq), 5, surface=True)
    assert ei.value.code == esdg.ESDG_EINVAL
    p.close()
    srv.close()


@pytest.mark.parametrize("rule,N", [("symmetric", 4), ("collapsed", 3)])
def test_weight_adjusted_with_walls_matches_oracle(rule, N):
    """The weight-adjusted inverse in a walled box (reflective walls, Sec. 2.9):
    right-hand side FP64 at 1e-12 and FP32 at 5e-5 against the oracle."""
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL, Solver
    w = W.DAM
    for precision, tol in (("fp64", 1e-12), ("fp32", 5e-5)):
        s = Solver(N, 6, 5, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, rule=rule, walls=True, mass=WA)
        o = Oracle(N, 6, 5, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, rule=rule, walls=True, mass=WA)
        xb, yb = s.points(ESDG_POINTS_NODAL)
        s.set_bathymetry(w.bathymetry(xb, yb))
        xo, yo = o.points("nodal")
        o.set_bathymetry(w.bathymetry(xo, yo))
        u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 50 + N)
        s.set_state(u)
        got = s.rhs(0.0).cpu().numpy()
        want = o.rhs(u, 0.0)
        assert _rel(got, want) < tol, precision
        if precision == "fp32":
            check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0), c_modal(o.Np, o.Nq, o.Nfq, wadg=True))
        s.close()
