"""Failure detection on the GPU without a fault: the stage kernels' bounded
wait on their bulk copies gives up, reports ESDG_ETIMEOUT through the status
word, and leaves the context usable (a solve right after it is exact)."""

import time

import numpy as np
import pytest

from oracle import Oracle
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


def test_bounded_wait_gives_up_and_reports_timeout():
    from paper_2005_02516_gb300 import esdg
    lib = esdg.load_library()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    rc = lib.esdg_selftest_wait_timeout(stream.cuda_stream)
    el = time.perf_counter() - t0
    assert rc == esdg.ESDG_ETIMEOUT
    assert 0.1 < el < 30.0          # the wait's limit is about a second of SM cycles
    # the device and a new context work normally afterwards
    w = W.LAKE_BUMP
    s = esdg.Solver(2, 5, 4, precision="fp32", warp=0.05, rule="symmetric")
    o = Oracle(2, 5, 4, ax=0.05, ay=0.05, rule="symmetric")
    xb, yb = s.points(esdg.ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    u = random_modal_state(o.K, o.Np, seed=W.BASE_SEED + 90)
    s.set_state(u)
    got = s.rhs(0.0).cpu().numpy()
    want = o.rhs(u, 0.0)
    assert np.linalg.norm(got - want) < 5e-5 * np.linalg.norm(want)
    s.close()
