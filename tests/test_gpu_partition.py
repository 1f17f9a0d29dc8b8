"""The element partition of one solve on the GPU: the blocks of a partition run
as separate contexts on one device, their halos exchanged by device copies
after the projection and after every RK stage (the exchange a multi-GPU run
makes through NCCL), and the result is compared with the same solve on one
context.

Each block's kernels see, element by element, exactly the inputs of the
single-domain run (its own records and geometry, its neighbours' face traces
in the ghost records), so the states must agree bit for bit, in FP64 and FP32; the
entropy and mass summed over blocks agree with the single-domain diagnostics
up to summation order (1e-12).  The single-domain path is held to the oracle
by the parity tests.
"""

import dataclasses

import numpy as np
import pytest

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


def _solver(w, precision, partition=None, method="modal", walls=False):
    from paper_2005_02516_gb300 import esdg
    s = esdg.Solver(w.N, w.nx, w.ny, precision=precision, warp=w.warp, g=w.g, cfl=w.cfl, rule=w.rule,
                    method=method, walls=walls, partition=partition)
    xb, yb = s.points(esdg.ESDG_POINTS_NODAL)
    xq, yq = s.points(esdg.ESDG_POINTS_VOLQ)
    s.init_state(w.bathymetry(xb, yb), w.initial(xq, yq))
    return s


CASES = [
    # (workload, px, py, method, walls)
    (dataclasses.replace(W.scaled(W.DAM, 12, 10), rule="symmetric"), 2, 1, "modal", False),
    (dataclasses.replace(W.scaled(W.DAM, 12, 10), rule="symmetric"), 2, 2, "modal", False),
    (dataclasses.replace(W.scaled(W.MMS, 9, 8, N=3), forcing="none"), 3, 2, "modal", False),
    (dataclasses.replace(W.scaled(W.DAM, 11, 9), rule="symmetric"), 2, 3, "modal", True),
    (W.scaled(W.LAKE_BUMP, 10, 8), 2, 2, "sbp", False),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("w,px,py,method,walls", CASES)
def test_partitioned_solve_equals_single_domain(w, px, py, method, walls, precision):
    from paper_2005_02516_gb300 import esdg
    from paper_2005_02516_gb300 import partition as P
    one = _solver(w, precision, method=method, walls=walls)
    dt = one.dt()
    nsteps = 7
    one.step(nsteps, dt, 0.0)
    want = one.get_state()
    S1, M1, _ = one.entropy(nsteps * dt, rate=False)
    parts = list(range(px * py))
    blocks, exs, maps = [], [], []
    for q in parts:
        s = _solver(w, precision, partition=(px, py, q), method=method, walls=walls)
        L = esdg.partition_layout(s.lib, s.h)
        ex = P.HaloExchange(P.halo_plan(L), L["trace_bytes"], s.halo_pack, s.halo_unpack)
        blocks.append(s)
        exs.append(ex)
        maps.append(L)
    # whole steps and single stages are refused on a block with ghosts
    with pytest.raises(esdg.EsdgError) as ei:
        blocks[0].step(1, dt, 0.0)
    assert ei.value.code == esdg.ESDG_ESTATE
    t = P.step_local(blocks, exs, parts, 3, dt, 0.0)
    t = P.step_local(blocks, exs, parts, nsteps - 3, dt, t)
    assert abs(t - nsteps * dt) < 1e-15
    got = np.full_like(want, np.nan)
    S, M = 0.0, 0.0
    for s, L in zip(blocks, maps):
        got[:, L["owned_gid"]] = s.get_state()
        Sq, Mq, _ = s.entropy(t, rate=False)
        S, M = S + Sq, M + Mq
    assert not np.isnan(got).any()
    assert np.array_equal(got, want), np.abs(got - want).max()
    assert abs(S - S1) <= 1e-12 * abs(S1) and abs(M - M1) <= 1e-12 * abs(M1)
    for s in blocks:
        s.close()
    one.close()


def test_halo_pack_and_unpack_move_face_traces():
    """esdg_halo_pack gathers the listed faces' traces (the N+1 node records of
    face f of element e; zeros for an entry out of range); esdg_halo_unpack
    writes traces into ghost faces, skipping entries out of range (that the
    written traces are the ones the interface flux reads is the bit-for-bit
    test above)."""
    from paper_2005_02516_gb300 import esdg
    w = dataclasses.replace(W.scaled(W.DAM, 8, 6), rule="symmetric")
    s = _solver(w, "fp32", partition=(2, 1, 0))
    L = esdg.partition_layout(s.lib, s.h)
    s.project()
    tb = L["trace_bytes"]
    assert tb == 4 * 4 * (w.N + 1)
    faces = torch.tensor([0, 4 * 3 + 2, 4 * (L["K"] - 1) + 1, 4 * (L["K"] + 5), 4 * 2 + 3, -1], dtype=torch.int32,
                         device="cuda")
    out = torch.full((faces.numel() * tb,), 7, dtype=torch.uint8, device="cuda")
    s.halo_pack(faces, out)
    tr = out.view(faces.numel(), tb)
    assert tr[0].any() and tr[1].any() and tr[2].any()
    assert not tr[3].any() and not tr[4].any() and not tr[5].any()
    assert not torch.equal(tr[0], tr[1])
    # unpack into the first ghost's faces and skip out-of-range entries
    dst = torch.tensor([0, 4 * 0 + 2, 4 * L["nghost"], -1], dtype=torch.int32, device="cuda")
    s.halo_unpack(out[:4 * tb], dst)
    s.check()
    s.close()
