"""The allocation-free entropy diagnostic (esdg_entropy_noalloc) against the
regular one (esdg_entropy), through the C ABI.

Callers that cannot allocate device memory while they run (an arena or pool
that forbids new allocations, a loop that must not call cudaMalloc) use the
variant whose scratch is a file-scope static device array.  Its results must
agree with esdg_entropy, whose scratch lives in the context's device buffer,
up to summation order (relative 1e-12), on two calls in a row: the second
call reuses the array the first call left behind.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _solver(precision):
    import os
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_02516_gb300 import esdg, workloads as W
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    w = W.DAM
    s = esdg.Solver(3, 12, 10, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl)
    xb, yb = s.points(esdg.ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    s.set_state(W.random_modal_state(s.K, s.Np, seed=W.BASE_SEED + 99))
    return s


def _noalloc(s, u_dev=None):
    S, M = ctypes.c_double(), ctypes.c_double()
    ptr = None if u_dev is None else u_dev.data_ptr()
    rc = s.lib.esdg_entropy_noalloc(s.h, ptr, ctypes.byref(S), ctypes.byref(M))
    assert rc == 0, s.lib.esdg_last_error(s.h)
    return S.value, M.value


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_entropy_matches_entropy_twice(precision):
    s = _solver(precision)
    S_ref, M_ref, _ = s.entropy(0.0, rate=False)
    for _ in range(2):
        S, M = _noalloc(s)
        assert abs(S - S_ref) <= 1e-12 * abs(S_ref)
        assert abs(M - M_ref) <= 1e-12 * abs(M_ref)
    # an explicit device state (after one step it differs from the first)
    u0 = torch.from_numpy(s.get_state()).cuda()
    s.step(1)
    S1_ref, M1_ref, _ = s.entropy(0.0, rate=False)
    S1, M1 = _noalloc(s)
    assert abs(S1 - S1_ref) <= 1e-12 * abs(S1_ref)
    S0, M0 = _noalloc(s, u0)
    assert abs(S0 - S_ref) <= 1e-12 * abs(S_ref)
    assert abs(M0 - M_ref) <= 1e-12 * abs(M_ref)
    assert np.isfinite([S1, M1]).all()
    s.close()


def test_noalloc_refuses_host_memory():
    # a host array handed in as the state would be read by the kernel as a
    # device address; the entry point refuses it before any launch
    s = _solver("fp64")
    S_ref, M_ref, _ = s.entropy(0.0, rate=False)
    host = np.ascontiguousarray(s.get_state())
    S, M = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    rc = s.lib.esdg_entropy_noalloc(s.h, host.ctypes.data_as(ctypes.c_void_p), ctypes.byref(S), ctypes.byref(M))
    from paper_2005_02516_gb300 import esdg
    assert rc == esdg.ESDG_EINVAL
    assert b"device memory" in s.lib.esdg_last_error(s.h)
    assert S.value == -1.0 and M.value == -1.0
    # the context is still usable afterwards
    S2, M2 = _noalloc(s)
    assert abs(S2 - S_ref) <= 1e-12 * abs(S_ref)
    s.close()
