"""GPU parity of the L2-error diagnostic (esdg_l2_error: the error measure of
the convergence study of Sec. 4.1 on the element's own volume rule) against
the oracle's l2_error_volq / SBPOracle.l2_error_volq on the same seeded state
and the same values at the volume points.  FP64 arithmetic on both sides:
relative 1e-12 per field."""

import ctypes

import numpy as np
import pytest

from oracle import Oracle
from oracle.sbp import SBPOracle
from paper_2005_02516_gb300 import workloads as W
from paper_2005_02516_gb300.workloads import random_modal_state

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


def _exact(x, y):
    """A smooth field per component, different for each."""
    return np.stack([2.0 + 0.3 * np.sin(np.pi * (x + y)), 0.5 * np.cos(np.pi * x), -0.2 * np.sin(2 * np.pi * y)])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,nx,ny,rule,mass", [(1, 3, 5, "collapsed", "exact"), (3, 5, 4, "collapsed", "exact"),
                                               (4, 6, 5, "symmetric", "exact"),
                                               (4, 4, 3, "symmetric", "weight_adjusted"),
                                               (5, 3, 4, "symmetric", "exact")])
def test_l2_error_matches_oracle_modal(N, nx, ny, rule, mass, precision):
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ, Solver
    s = Solver(N, nx, ny, precision=precision, warp=0.05, rule=rule, mass=mass)
    o = Oracle(N, nx, ny, ax=0.05, ay=0.05, rule=rule, mass=mass)
    u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 90 + N)
    s.set_state(u)
    x, y = s.points(ESDG_POINTS_VOLQ)
    xo, yo = o.points("volq")
    assert np.allclose(x, xo, rtol=0, atol=1e-13) and np.allclose(y, yo, rtol=0, atol=1e-13)
    got = s.l2_error(_exact(x, y))
    want = o.l2_error_volq(u, _exact(xo, yo))
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (got, want)
    # the closed form of the pins: u_h = 0 against the constant c -> 2 c
    s.set_state(np.zeros_like(u))
    got0 = s.l2_error(np.stack([np.full((o.K, o.Nq), c) for c in (1.0, 2.0, 3.0)]))
    assert np.allclose(got0, [2.0, 4.0, 6.0], rtol=1e-12, atol=0)
    s.close()


@pytest.mark.parametrize("N", [2, 4])
def test_l2_error_matches_oracle_sbp(N):
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_VOLQ, Solver
    s = Solver(N, 5, 4, precision="fp64", warp=0.05, method="sbp")
    o = SBPOracle(N, 5, 4, ax=0.05, ay=0.05)
    rng = np.random.default_rng(W.BASE_SEED + 95 + N)
    u = np.stack([2.0 + 0.1 * rng.standard_normal((o.K, o.Nq)), 0.1 * rng.standard_normal((o.K, o.Nq)),
                  0.1 * rng.standard_normal((o.K, o.Nq))])
    s.set_state(u)
    x, y = s.points(ESDG_POINTS_VOLQ)
    got = s.l2_error(_exact(x, y))
    xo, yo = o.points("volq")
    want = o.l2_error_volq(u, _exact(xo, yo))
    assert np.all(np.abs(got - want) <= 1e-12 * np.abs(want)), (got, want)
    s.close()


def test_l2_error_refuses_host_memory():
    from paper_2005_02516_gb300 import esdg
    s = esdg.Solver(2, 4, 4, precision="fp64")
    host = np.zeros((3, s.K, s.Nq))
    err = (ctypes.c_double * 3)()
    assert s.lib.esdg_l2_error(s.h, host.ctypes.data, err) == esdg.ESDG_EINVAL
    s.close()
