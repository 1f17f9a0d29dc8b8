"""GPU parity of the DG-SBP scheme (ESDG_METHOD_SBP, Sec. 3) against the
oracle's SBPOracle on the same seeded nodal inputs.

Tolerances as for the modal scheme: FP64 relative 1e-12 on the right-hand
side and on the state after every step; FP32 right-hand side 5e-5 relative,
FP32 state after the configured steps 1e-5.
"""

import dataclasses

import numpy as np
import pytest

from oracle.esdg import mms_sine_forcing
from oracle.sbp import SBPOracle
from paper_2005_02516_gb300 import workloads as W

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


def _pair(w, precision, N, nx, ny, lf=True):
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL, Solver
    s = Solver(N, nx, ny, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, lax_friedrichs=lf,
               forcing=w.forcing, method="sbp")
    o = SBPOracle(N, nx, ny, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, lf=lf,
                  forcing=mms_sine_forcing if w.forcing == "mms_sine" else None)
    xb, yb = s.points(ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    return s, o


def _state(w, o, seed, amp=0.02):
    """The workload's initial data at the SBP nodes plus seeded noise."""
    x, y = o.points("volq")
    q = np.array(w.initial(x, y), dtype=np.float64)
    if w.surface_init:
        q[0] = q[0] - o.bq
    rng = np.random.default_rng(seed)
    return q + amp * rng.standard_normal(q.shape)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


from _bounds import c_sbp, check_fp32_rhs, check_state  # noqa: E402


CASES = [
    # (workload, N, nx, ny): affine and curved meshes, the manufactured
    # solution's forcing, ragged element counts
    (W.LAKE_BUMP, 2, 8, 8),
    (dataclasses.replace(W.LAKE_BUMP, warp=0.05), 1, 5, 3),
    (W.MMS, 3, 5, 4),
    (W.MMS, 4, 3, 5),
    (dataclasses.replace(W.LAKE_BUMP, warp=0.05), 5, 4, 3),
]


@pytest.mark.parametrize("lf", [True, False])
@pytest.mark.parametrize("w,N,nx,ny", CASES)
def test_sbp_rhs_matches_oracle(w, N, nx, ny, lf):
    for precision, tol in (("fp64", 1e-12), ("fp32", 5e-5)):
        s, o = _pair(w, precision, N, nx, ny, lf)
        u = _state(w, o, seed=W.BASE_SEED + 60 + N)
        s.set_state(u)
        got = s.rhs(0.17).cpu().numpy()
        want = o.rhs(u, 0.17)
        assert _rel(got, want) < tol, precision
        if precision == "fp32":
            check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.17), c_sbp(o.Nq))
        s.close()


@pytest.mark.parametrize("N", [2, 4])
def test_sbp_steps_match_oracle(N):
    """The manufactured solution on a curved 6 x 5 mesh: FP64 per step at 1e-12
    for 15 steps (init_state included), FP32 after the same steps at 1e-5."""
    w = W.scaled(W.MMS, 6, 5, N=N)
    s64, o = _pair(w, "fp64", N, 6, 5)
    s32, _ = _pair(w, "fp32", N, 6, 5)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s64.points(ESDG_POINTS_VOLQ)
    s64.init_state(None, w.initial(xs, ys))
    xq, yq = o.points("volq")
    u = o.init_state(w.initial(xq, yq))
    assert _rel(s64.get_state(), u) < 1e-15
    s32.set_state(u)
    res = np.zeros_like(u)
    t, dt = 0.0, o.dt()
    for n in range(15):
        u, res, t = o.step(u, res, t, dt)
        s64.step(1, dt, t - dt)
        assert _rel(s64.get_state(), u) < 1e-12, n
    s32.step(15, dt, 0.0)
    check_state(s32.get_state(), u, 1e-5)


def test_sbp_lake_at_rest_entropy_and_mass_on_gpu():
    """Lake at rest (surface init) stays at rest; with the EC flux alone the
    entropy rate from esdg_entropy vanishes; entropy and mass match the
    oracle's nodal sums; mass is conserved over steps."""
    w = dataclasses.replace(W.LAKE_BUMP, warp=0.05)
    s, o = _pair(w, "fp64", 3, 6, 6)
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ
    xs, ys = s.points(ESDG_POINTS_VOLQ)
    s.init_state(None, np.stack([2.0 + 0 * xs, 0 * xs, 0 * xs]), surface=True)
    assert np.abs(s.rhs().cpu().numpy()).max() < 1e-12
    s2, o2 = _pair(w, "fp64", 3, 6, 6, lf=False)
    u = _state(w, o2, seed=11)
    s2.set_state(u)
    S, M, R = s2.entropy(0.0)
    terms = o2.entropy_rate_terms(u, o2.rhs(u))
    assert abs(R) < 1e-12 * np.abs(terms).sum()
    assert abs(S - o2.entropy(u)) < 1e-12 * abs(S)
    assert abs(M - o2.mass(u)) < 1e-12 * abs(M)
    s2.step(5)
    assert abs(s2.entropy(0.0, rate=False)[1] - M) < 1e-12 * abs(M)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sbp_full_size_sampled_rhs(precision):
    """The smoothed dam break at full size (N=4, K=131072 curved, 22 SBP nodes
    per element): the right-hand side on every 997th element (and the last)
    against the oracle element by element; FP64 at 1e-12, FP32 entry by entry
    within the first-order FP32 bound c u mag (tests/_bounds.py)."""
    w = W.DAM
    s, o = _pair(w, precision, w.N, w.nx, w.nx)
    x, y = o.points("volq")
    u = o.init_state(w.initial(x, y))
    s.set_state(u)
    ks = np.unique(np.concatenate([np.arange(0, o.K, 997), [o.K - 1]]))
    got = s.rhs(0.0).cpu().numpy()[:, ks]
    want = o.rhs_elements(u, ks)
    if precision == "fp64":
        assert _rel(got, want) < 1e-12
    else:
        check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0, elems=ks), c_sbp(o.Nq))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sbp_step_host_equals_set_step_copy(precision):
    w = W.scaled(W.MMS, 5, 4, N=3)
    s, o = _pair(w, precision, 3, 5, 4)
    u = _state(w, o, seed=W.BASE_SEED + 71)
    host = torch.empty((3, o.K, o.Nq), dtype=torch.float64, pin_memory=True).numpy()
    out = torch.empty((3, o.K, o.Nq), dtype=torch.float64, pin_memory=True).numpy()
    host[:] = u
    dt = o.dt()
    s.step_host(host, 3, dt, 0.0, out=out)
    s.set_state(u)
    s.step(3, dt, 0.0)
    assert np.array_equal(out, s.get_state())


def test_sbp_is_refused_by_ensembles_and_served_fp32():
    """Ensembles (and so served FP32 requests) run the modal scheme only;
    served FP64 requests take the DG-SBP method (test_gpu_serving.py)."""
    from paper_2005_02516_gb300 import esdg
    s = esdg.Solver(2, 8, 8, precision="fp32", method="sbp")
    with pytest.raises(esdg.EsdgError) as ei:
        esdg.Ensemble([s])
    assert ei.value.code == esdg.ESDG_EINVAL
    s.close()
    p = esdg.Problem(2, 8, 8, precision="fp32", method="sbp")
    xb, yb = p.points(esdg.ESDG_POINTS_NODAL)
    xq, yq = p.points(esdg.ESDG_POINTS_VOLQ)
    srv = esdg.Server(hbm_budget_bytes=1 << 30)
    with pytest.raises(esdg.EsdgError) as ei:
        srv.submit(p, W.LAKE_BUMP.bathymetry(xb, yb), W.LAKE_BUMP.initial(xq, yq), 5, surface=True)
    assert ei.value.code == esdg.ESDG_EINVAL
    p.close()
    srv.close()
