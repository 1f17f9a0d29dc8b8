"""The volume-kernel cost comparison of Sec. 5.4 on the CPU: the oracle's
DG and ESDG volume terms against what the definitions fix, and the library's
host implementation (esdg_volume_kernel_host) against the oracle."""

import numpy as np
import pytest

from oracle.swe import ec_flux, physical_flux
from oracle.volume import volume_dg, volume_esdg
from paper_2005_02516_gb300 import workloads as W


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_constant_state_esdg_equals_dg():
    # f_S(u, u) = f(u) (consistency, Definition 2.1): with the same state at
    # every node both kernels reduce to Q^x f^x + Q^y f^y
    Qx, Qy, u = W.volume_ratio_inputs(9, 3, seed=1)
    u[:] = u[:, :, :1]
    assert _rel(volume_esdg(Qx, Qy, u, 1.3), volume_dg(Qx, Qy, u, 1.3)) < 1e-14


def test_skew_operators_give_zero_total_esdg():
    # F^i is symmetric in its node pair, so for skew-symmetric Q the sum of all
    # rows of (Q o F) 1 vanishes (the flux-differencing conservation property)
    Qx, Qy, u = W.volume_ratio_inputs(12, 4, seed=2)
    Qx, Qy = Qx - Qx.T, Qy - Qy.T
    r = volume_esdg(Qx, Qy, u, 1.0)
    scale = np.abs(r).sum(axis=2)
    assert np.all(np.abs(r.sum(axis=2)) < 1e-13 * scale)


def test_identity_operators_closed_form():
    Qx, Qy, u = W.volume_ratio_inputs(7, 2, seed=3)
    eye = np.eye(7)
    fx, fy = physical_flux(u, 0.7)
    assert _rel(volume_dg(eye, eye, u, 0.7), fx + fy) < 1e-15
    assert _rel(volume_esdg(eye, eye, u, 0.7), fx + fy) < 1e-14
    assert _rel(volume_esdg(eye, 0 * eye, u, 0.7), fx) < 1e-14


def test_esdg_against_scalar_pair_loop():
    Qx, Qy, u = W.volume_ratio_inputs(4, 2, seed=4)
    g = 0.9
    want = np.zeros_like(u)
    for e in range(2):
        for j in range(4):
            for k in range(4):
                fx, fy = ec_flux(u[:, e, j], u[:, e, k], g)
                want[:, e, j] += Qx[j, k] * fx + Qy[j, k] * fy
    assert _rel(volume_esdg(Qx, Qy, u, g), want) < 1e-14


def test_dg_is_linear_in_the_operators():
    Qx, Qy, u = W.volume_ratio_inputs(6, 3, seed=5)
    A, B, _ = W.volume_ratio_inputs(6, 1, seed=6)
    lhs = volume_dg(Qx + A, Qy + B, u, 1.0)
    rhs = volume_dg(Qx, Qy, u, 1.0) + volume_dg(A, B, u, 1.0)
    assert _rel(lhs, rhs) < 1e-14


@pytest.mark.parametrize("n,K", [(1, 1), (3, 5), (17, 2), (40, 3)])
@pytest.mark.parametrize("kind", ["dg", "esdg"])
@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 2e-5)])
def test_library_host_kernel_matches_oracle(n, K, kind, dtype, tol):
    from paper_2005_02516_gb300 import esdg
    import os
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    Qx, Qy, u = W.volume_ratio_inputs(n, K, seed=10 + n)
    g = 1.0
    want = (volume_esdg if kind == "esdg" else volume_dg)(Qx, Qy, u, g)
    code = esdg.ESDG_VOLUME_ESDG if kind == "esdg" else esdg.ESDG_VOLUME_DG
    got = esdg.volume_kernel(code, Qx.astype(dtype), Qy.astype(dtype), u.astype(dtype), g)
    assert got.dtype == dtype
    assert _rel(got.astype(np.float64), want) < tol


@pytest.mark.parametrize("bad", [dict(n=0), dict(n=257), dict(K=0), dict(kind=2), dict(precision=5)])
def test_volume_kernel_rejects_bad_arguments(bad):
    from paper_2005_02516_gb300 import esdg
    lib = esdg.load_library()
    a = dict(kind=0, precision=esdg.ESDG_FP64, n=4, K=2)
    a.update(bad)
    buf = np.ones(3 * 2 * 300 * 300)
    rc = lib.esdg_volume_kernel_host(a["kind"], a["precision"], a["n"], a["K"], 1.0, buf.ctypes.data,
                                     buf.ctypes.data, buf.ctypes.data, buf.ctypes.data)
    assert rc == esdg.ESDG_EINVAL
