"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances.  FP64: relative 1e-12 on the right-hand side and on the state
after every step (both sides compute the same operator in different forms and
summation orders: eq. (dgform) literally on the oracle side, the split form of
Sec. 5.2 on the GPU).  FP32 right-hand side with FP64 RK accumulation:
relative 1e-5 on the state after the configured steps, in the L2 norm and
entry by entry against the largest entry; a single FP32 right-hand side is
held entry by entry to c u times the magnitude of the terms it sums (the
first-order FP32 error bound derived in tests/_bounds.py), and to 5e-5
relative in norm.
"""

import numpy as np
import pytest

from oracle import Oracle
from oracle.esdg import mms_sine_forcing
from paper_2005_02516_gb300 import workloads as W
from paper_2005_02516_gb300.workloads import random_modal_state
from _bounds import c_modal, check_fp32_rhs, check_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    from paper_2005_02516_gb300 import esdg
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()


def _solver(w, precision="fp64", lf=True, N=None, nx=None, ny=None, rule=None, walls=False):
    from paper_2005_02516_gb300.esdg import Solver
    N = w.N if N is None else N
    nx = w.nx if nx is None else nx
    ny = nx if ny is None else ny
    rule = w.rule if rule is None else rule
    s = Solver(N, nx, ny, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, lax_friedrichs=lf,
               forcing=w.forcing, rule=rule, walls=walls)
    o = Oracle(N, nx, ny, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, lf=lf,
               forcing=mms_sine_forcing if w.forcing == "mms_sine" else None, rule=rule, walls=walls)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL
    xb, yb = s.points(ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    return s, o


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


CASES = [
    # (workload, N, nx, ny) -- several tiles (8 elements per CTA) and ragged tails
    (W.LAKE_BUMP, 2, 8, 8),
    (W.LAKE_BUMP, 1, 5, 3),
    (W.MMS, 3, 5, 4),
    (W.MMS, 4, 3, 5),
    (W.DAM, 4, 6, 5),
    (W.DAM, 5, 4, 3),
]


RULES = ["collapsed", "symmetric"]


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("lf", [True, False])
@pytest.mark.parametrize("w,N,nx,ny", CASES)
def test_rhs_fp64_matches_oracle(w, N, nx, ny, lf, rule):
    s, o = _solver(w, "fp64", lf, N, nx, ny, rule)
    u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + N)
    s.set_state(u)
    t = 0.37
    got = s.rhs(t).cpu().numpy()
    want = o.rhs(u, t)
    assert _rel(got, want) < 1e-12
    assert _relmax(got, want) < 1e-12


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("w,N,nx,ny", CASES)
def test_rhs_fp32_matches_oracle(w, N, nx, ny, rule):
    s, o = _solver(w, "fp32", True, N, nx, ny, rule)
    u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 10 + N)
    s.set_state(u)
    got = s.rhs(0.1).cpu().numpy()
    want = o.rhs(u, 0.1)
    assert _rel(got, want) < 5e-5
    check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.1), c_modal(o.Np, o.Nq, o.Nfq))


def test_steps_fp64_config1_match_oracle_every_step():
    """Lake at rest plus a bump (N=2, K=128 affine): per-step parity
    for 20 steps at relative 1e-12."""
    w = W.LAKE_BUMP
    s, o = _solver(w, "fp64")
    xq, yq = o.points("volq")
    u = o.init_state(w.initial(xq, yq), surface=True)
    s.set_state(u)
    res = np.zeros_like(u)
    t, dt = 0.0, o.dt()
    for n in range(20):
        u, res, t = o.step(u, res, t, dt)
        s.step(1, dt, t - dt)
        assert _rel(s.get_state(), u) < 1e-12, n


def test_init_state_matches_oracle():
    w = W.MMS
    s, o = _solver(w, "fp64", N=3, nx=6)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s.points(ESDG_POINTS_VOLQ)
    s.init_state(None, w.initial(xs, ys))
    xo, yo = o.points("volq")
    uo = o.init_state(w.initial(xo, yo))
    assert _rel(s.get_state(), uo) < 1e-13


@pytest.mark.parametrize("rule", RULES)
def test_fp32_after_configured_steps_config1(rule):
    """Lake at rest plus a bump (N=2, K=128) for all 200 configured steps:
    FP32 RHS with FP64 accumulation
    within relative 1e-5 of the FP64 oracle; FP64 within 1e-12."""
    w = W.LAKE_BUMP
    s64, o = _solver(w, "fp64", rule=rule)
    s32, _ = _solver(w, "fp32", rule=rule)
    xq, yq = o.points("volq")
    u0 = o.init_state(w.initial(xq, yq), surface=True)
    u, _ = o.run(u0, w.steps)
    for s, tol in [(s64, 1e-12), (s32, 1e-5)]:
        s.set_state(u0)
        s.step(w.steps)
        check_state(s.get_state(), u, tol)


@pytest.mark.parametrize("rule", RULES)
def test_lake_at_rest_and_entropy_on_gpu(rule):
    """Theorem 2.2 on the GPU path: a lake at rest stays at rest, and with the
    EC flux alone the semi-discrete entropy rate vanishes.  Curved mesh,
    periodic continuous bathymetry, no forcing."""
    import dataclasses
    w = dataclasses.replace(W.LAKE_BUMP, warp=0.05, rule=rule)
    s, o = _solver(w, "fp64", lf=True, N=3, nx=6)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s.points(ESDG_POINTS_VOLQ)
    q = np.stack([2.0 + 0 * xs, 0 * xs, 0 * xs])
    s.init_state(None, q, surface=True)
    r = s.rhs().cpu().numpy()
    assert np.abs(r).max() < 1e-12
    s2, o2 = _solver(w, "fp64", lf=False, N=3, nx=6)
    u = random_modal_state(o2.K, o2.Np, seed=7)
    s2.set_state(u)
    S, M, R = s2.entropy(0.0)
    terms = o2.entropy_rate_terms(u, o2.rhs(u))
    assert abs(R) < 1e-12 * np.abs(terms).sum()
    assert abs(S - o2.entropy(u)) < 1e-12 * abs(S)
    assert abs(M - o2.mass(u)) < 1e-12 * abs(M)
    s2.step(5)
    S5, M5, _ = s2.entropy(0.0, rate=False)
    assert abs(M5 - M) < 1e-12 * abs(M)


@pytest.mark.parametrize("rule", RULES)
def test_lake_at_rest_fp32_on_gpu(rule):
    """The FP32 path keeps a lake at rest over curved, continuous bathymetry to
    FP32 roundoff of the pressure terms (their size here is about g h H / dx *
    N^2 ~ 1e2, so roundoff ~1e-5): the kernel's free surface relative to each
    element's first node is exact by Q_h 1 = 0 and leaves only the projection's
    roundoff."""
    import dataclasses
    w = dataclasses.replace(W.LAKE_BUMP, warp=0.05, rule=rule)
    s, o = _solver(w, "fp32", lf=True, N=3, nx=6)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s.points(ESDG_POINTS_VOLQ)
    s.init_state(None, np.stack([2.0 + 0 * xs, 0 * xs, 0 * xs]), surface=True)
    r = s.rhs().cpu().numpy()
    assert np.abs(r).max() < 1e-4, np.abs(r).max()
    xo, yo = o.points("volq")
    uo = o.init_state(np.stack([2.0 + 0 * xo, 0 * xo, 0 * xo]), surface=True)
    # the exact right-hand side is zero; entry by entry within the FP32 bound
    check_fp32_rhs(r, 0.0 * r, o.rhs_term_magnitude(uo), c_modal(o.Np, o.Nq, o.Nfq))
    s.step(20)
    u = s.get_state()
    s64, _ = _solver(w, "fp64", lf=True, N=3, nx=6)
    s64.init_state(None, np.stack([2.0 + 0 * xs, 0 * xs, 0 * xs]), surface=True)
    u0 = s64.get_state()
    check_state(u, u0, 1e-5)


def test_nonpositive_depth_is_reported_not_faulted():
    from paper_2005_02516_gb300.esdg import EsdgError, ESDG_ENONPOSITIVE
    w = W.LAKE_BUMP
    s, o = _solver(w, "fp64")
    u = random_modal_state(o.K, o.Np, seed=3)
    u[0] *= -1.0
    s.set_state(u)
    with pytest.raises(EsdgError) as ei:
        s.rhs()
    assert ei.value.code == ESDG_ENONPOSITIVE
    # the context stays usable
    u = random_modal_state(o.K, o.Np, seed=3)
    s.set_state(u)
    s.rhs()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_config3_sampled_rhs(precision):
    """Smoothed dam break at full size (N=4, K=131072 curved, the 16-point
    symmetric volume rule, as benchmarked): the right-hand side on
    sampled elements (every 997th, plus the first and last) against the
    oracle computed element by element, in the launch configuration the
    benchmark uses.  FP64: relative 1e-12 in norm and max norm.  FP32: every
    sampled entry within the first-order FP32 bound c u mag (tests/_bounds.py),
    mag the magnitude of the terms that entry sums; the state is at rest away
    from the front, where du/dt is a cancellation of pressure terms of size
    g h^2 / dx, so a bound relative to du/dt itself would not be one."""
    w = W.DAM
    s, o = _solver(w, precision)
    xo, yo = o.points("volq")
    u = o.init_state(w.initial(xo, yo))
    s.set_state(u)
    ks = np.unique(np.concatenate([np.arange(0, o.K, 997), [o.K - 1]]))
    got = s.rhs(0.0).cpu().numpy()[:, ks]
    want = o.rhs_elements(u, ks)
    if precision == "fp64":
        assert _rel(got, want) < 1e-12
        assert _relmax(got, want) < 1e-12
    else:
        check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0, elems=ks), c_modal(o.Np, o.Nq, o.Nfq))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_collapsed_rule_sampled_rhs(precision):
    """The same full-size workload with the collapsed (N+1)^2 = 25-point
    volume rule (the bench's collapsed-rule line; 675 non-zero pairs of Q_skew
    per element, ordered pairs in both kernels, the FP64 path's pieces
    schedule): the right-hand side on every 997th element (plus the last)
    against the oracle element by element, FP64 at relative 1e-12, FP32 within
    the first-order bound of each entry."""
    w = W.DAM
    s, o = _solver(w, precision, rule="collapsed")
    xo, yo = o.points("volq")
    u = o.init_state(w.initial(xo, yo))
    s.set_state(u)
    ks = np.unique(np.concatenate([np.arange(0, o.K, 997), [o.K - 1]]))
    got = s.rhs(0.0).cpu().numpy()[:, ks]
    want = o.rhs_elements(u, ks)
    if precision == "fp64":
        assert _rel(got, want) < 1e-12
        assert _relmax(got, want) < 1e-12
    else:
        check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0, elems=ks), c_modal(o.Np, o.Nq, o.Nfq))


# ---- reflective walls (Sec. 2.9) -----------------------------------------------
WALL_CASES = [(W.DAM, 4, 6, 5, "symmetric"), (W.DAM, 3, 5, 4, "collapsed"), (W.LAKE_BUMP, 2, 7, 3, "symmetric"),
              (W.DAM, 5, 4, 3, "symmetric")]


@pytest.mark.parametrize("lf", [True, False])
@pytest.mark.parametrize("w,N,nx,ny,rule", WALL_CASES)
def test_walls_rhs_matches_oracle(w, N, nx, ny, rule, lf):
    for precision, tol in (("fp64", 1e-12), ("fp32", 5e-5)):
        s, o = _solver(w, precision, lf, N, nx, ny, rule, walls=True)
        u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 20 + N)
        s.set_state(u)
        got = s.rhs(0.2).cpu().numpy()
        want = o.rhs(u, 0.2)
        assert _rel(got, want) < tol, precision
        if precision == "fp32":
            check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.2), c_modal(o.Np, o.Nq, o.Nfq))
        s.close()


def test_walls_steps_and_lake_at_rest_on_gpu():
    """The smoothed dam break in a walled box (its bump is not periodic):
    FP64 steps match the oracle at 1e-12 per step, FP32 at 1e-5 after 20
    steps; a lake at rest over the bump stays at rest on both paths."""
    w = W.scaled(W.DAM, 6, 5)
    s64, o = _solver(w, "fp64", walls=True)
    s32, _ = _solver(w, "fp32", walls=True)
    xq, yq = o.points("volq")
    u = o.init_state(w.initial(xq, yq))
    s64.set_state(u)
    s32.set_state(u)
    res = np.zeros_like(u)
    t, dt = 0.0, o.dt()
    for n in range(20):
        u, res, t = o.step(u, res, t, dt)
        s64.step(1, dt, t - dt)
        assert _rel(s64.get_state(), u) < 1e-12, n
    s32.step(20, dt, 0.0)
    check_state(s32.get_state(), u, 1e-5)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    for s in (s64, s32):
        xs, ys = s.points(ESDG_POINTS_VOLQ)
        s.init_state(None, np.stack([1.5 + 0 * xs, 0 * xs, 0 * xs]), surface=True)
        # FP32: roundoff of O(Nh) flux terms of size g h^2 / dx ~ 10 per entry
        assert np.abs(s.rhs().cpu().numpy()).max() < (1e-12 if s is s64 else 1e-4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_host_equals_set_step_copy(precision):
    """esdg_step_host (the device reads the pinned host state and writes the
    result back) gives exactly the state of set_state + step + copy_state."""
    from paper_2005_02516_gb300.esdg import EsdgError, ESDG_EINVAL
    w = W.scaled(W.DAM, 7, 5)
    s, o = _solver(w, precision)
    u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 31)
    host = torch.empty((3, o.K, o.Np), dtype=torch.float64, pin_memory=True).numpy()
    out = torch.empty((3, o.K, o.Np), dtype=torch.float64, pin_memory=True).numpy()
    host[:] = u
    dt = o.dt()
    _, t = s.step_host(host, 3, dt, 0.0, out=out)
    assert abs(t - 3 * dt) < 1e-15
    s2, _ = _solver(w, precision)
    s2.set_state(u)
    s2.step(3, dt, 0.0)
    assert np.array_equal(out, s2.get_state())
    assert np.array_equal(host, u)                     # the input is left alone
    # in place (a host-state call always starts from the host state, like
    # set_state), and the device state follows
    host[:] = out
    s.step_host(host, 2, dt, 3 * dt)
    s2.set_state(out)
    s2.step(2, dt, 3 * dt)
    assert np.array_equal(host, s2.get_state()) and np.array_equal(s.get_state(), host)
    # pageable host memory is refused, the context stays usable
    with pytest.raises(EsdgError) as ei:
        s.step_host(np.array(u), 1, dt)
    assert ei.value.code == ESDG_EINVAL
    s.step(1, dt)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_is_exact(precision):
    """Checkpoint / resume: the state u alone restarts LSRK45 (its first
    stage has A = 0, so the residual carries nothing across steps).  Ten steps
    in one run equal five steps, esdg_copy_state, a new context,
    esdg_set_state and five more steps, to rounding: the resumed run projects
    its first u~ in the projection kernel rather than at the end of a stage
    kernel, whose compiled arithmetic may round differently."""
    w = W.scaled(W.MMS, 6, 5)
    s1, o = _solver(w, precision, nx=6, ny=5)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s1.points(ESDG_POINTS_VOLQ)
    q = w.initial(xs, ys)
    s1.init_state(None, q)
    dt = o.dt()
    s1.step(10, dt, 0.0)
    u10 = s1.get_state()
    s2, _ = _solver(w, precision, nx=6, ny=5)
    s2.init_state(None, q)
    s2.step(5, dt, 0.0)
    ck = s2.get_state()
    s2.close()
    s3, _ = _solver(w, precision, nx=6, ny=5)
    s3.set_state(ck)
    s3.step(5, dt, 5 * dt)
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.linalg.norm(s3.get_state() - u10) <= tol * np.linalg.norm(u10)
