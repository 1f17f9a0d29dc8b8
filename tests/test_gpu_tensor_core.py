"""The FP32 path with its dense contractions on the tensor cores (dense =
"tensor": Vq, Vq^T W J, Vh and the lift Vh^T as tcgen05 MMAs with TF32
operands split into two parts) against the FP64 oracle and against the same
path on the FP32 pipes.

Tolerances: a right-hand side entry by entry within c u times the magnitude
of its terms, c from tests/_bounds.c_modal_tc (the FP32 bound plus the
split-TF32 products); states after the configured steps within the 1e-5
relative bar (L2 and max norm) of the FP64 path, itself held to the oracle at
1e-12 per step by the parity tests.
"""

import numpy as np
import pytest

from oracle import Oracle
from oracle.esdg import mms_sine_forcing
from paper_2005_02516_gb300 import workloads as W
from paper_2005_02516_gb300.workloads import random_modal_state
from _bounds import c_modal_tc, check_fp32_rhs, check_state

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


def _solver(w, N, nx, ny, rule, precision="fp32", dense="tensor", walls=False):
    from paper_2005_02516_gb300.esdg import Solver, ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    s = Solver(N, nx, ny, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, forcing=w.forcing, rule=rule,
               walls=walls, dense=dense)
    xb, yb = s.points(ESDG_POINTS_NODAL)
    s.set_bathymetry(w.bathymetry(xb, yb))
    return s


# degrees with the tensor-core form: Np <= 16 and Nq <= 16
SUPPORTED = [("symmetric", 1), ("symmetric", 2), ("symmetric", 3), ("symmetric", 4),
             ("collapsed", 1), ("collapsed", 2), ("collapsed", 3)]


@pytest.mark.parametrize("w", [W.DAM, W.MMS], ids=["dam", "mms_forcing"])
@pytest.mark.parametrize("rule,N", SUPPORTED)
def test_tensor_core_rhs_matches_oracle(rule, N, w):
    """One right-hand side (MODE 0: volume, interface, lift on the tensor
    cores, inverse mass) on a random state, ragged batch tail included."""
    nx, ny = 7, 5   # K = 70: a ragged last batch of 4 elements
    s = _solver(w, N, nx, ny, rule)
    o = Oracle(N, nx, ny, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl,
               forcing=mms_sine_forcing if w.forcing == "mms_sine" else None, rule=rule)
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    u = random_modal_state(o.K, o.Np, seed=11 + N)
    s.set_state(u)
    got = s.rhs(0.3).cpu().numpy()
    want = o.rhs(u, 0.3)
    check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.3), c_modal_tc(o.Np, o.Nq, o.Nfq))
    s.close()


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("rule,N", [("symmetric", 4), ("collapsed", 3), ("symmetric", 2)])
def test_tensor_core_steps_match_fp64_path(rule, N, walls):
    """Whole steps (MODE 2 projection, then RK stages with the projection of
    every new state on the tensor cores) against the FP64 path, and against
    the same steps on the FP32 pipes."""
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    w = W.DAM
    states = {}
    for name, prec, dense in (("fp64", "fp64", "auto"), ("simt", "fp32", "simt"), ("tensor", "fp32", "tensor")):
        s = _solver(w, N, 12, 10, rule, precision=prec, dense=dense, walls=walls)
        xb, yb = s.points(ESDG_POINTS_NODAL)
        xq, yq = s.points(ESDG_POINTS_VOLQ)
        s.init_state(w.bathymetry(xb, yb), w.initial(xq, yq))
        s.step(12, s.dt(), 0.0)
        states[name] = s.get_state()
        s.close()
    check_state(states["tensor"], states["fp64"], 1e-5)
    check_state(states["tensor"], states["simt"], 1e-5)


def test_tensor_core_ensemble_runs_on_fp32_pipes():
    """An ensemble accepts contexts built with dense = "tensor": its kernel
    applies the dense operators on the FP32 pipes, from the operator copy such
    a context keeps in that layout, and only the first entropy projection runs
    through each member's own (tensor-core) kernel.  The result agrees with the
    ensemble of the same contexts built with dense = "simt" within the FP32
    state bar."""
    from paper_2005_02516_gb300 import esdg
    from paper_2005_02516_gb300.esdg import ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    w = W.DAM
    out = {}
    for dense in ("simt", "tensor"):
        members = []
        for N, nx in ((4, 6), (2, 9), (3, 5)):
            s = esdg.Solver(N, nx, nx, precision="fp32", warp=w.warp, g=w.g, cfl=w.cfl, rule="symmetric",
                            dense=dense)
            xb, yb = s.points(ESDG_POINTS_NODAL)
            xq, yq = s.points(ESDG_POINTS_VOLQ)
            s.init_state(w.bathymetry(xb, yb), w.initial(xq, yq))
            members.append(s)
        ens = esdg.Ensemble(members)
        ens.step(7)
        out[dense] = [m.get_state() for m in members]
        ens.close()
        for m in members:
            m.close()
    for a, b in zip(out["tensor"], out["simt"]):
        check_state(a, b, 1e-5)


@pytest.mark.parametrize("kw", [dict(N=5, rule="symmetric"), dict(N=4, rule="collapsed"),
                                dict(N=3, rule="symmetric", precision="fp64"),
                                dict(N=3, rule="symmetric", mass="weight_adjusted")])
def test_tensor_core_refused_where_it_does_not_exist(kw):
    from paper_2005_02516_gb300 import esdg
    with pytest.raises(esdg.EsdgError) as ei:
        esdg.Solver(kw.pop("N"), 4, 4, precision=kw.pop("precision", "fp32"), dense="tensor", **kw)
    assert ei.value.code == esdg.ESDG_EINVAL


def test_tensor_core_full_size_sampled_rhs():
    """The smoothed dam break at full size (N = 4, K = 131072 curved, the
    16-point symmetric rule), the tensor-core form in its launch
    configuration: the right-hand side on sampled elements (every 997th,
    plus the first and last) against the oracle element by element, within
    the split-TF32 bound."""
    w = W.DAM
    s = _solver(w, w.N, w.nx, w.nx, w.rule)
    o = Oracle(w.N, w.nx, w.nx, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, rule=w.rule)
    xo, yo = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xo, yo))
    xq, yq = o.points("volq")
    u = o.init_state(w.initial(xq, yq))
    s.set_state(u)
    ks = np.unique(np.concatenate([np.arange(0, o.K, 997), [o.K - 1]]))
    got = s.rhs(0.0).cpu().numpy()[:, ks]
    want = o.rhs_elements(u, ks)
    check_fp32_rhs(got, want, o.rhs_term_magnitude(u, 0.0, elems=ks), c_modal_tc(o.Np, o.Nq, o.Nfq))
    s.close()
