"""The element partition of one solve (multi-GPU form of a single solve), on
the CPU: the partitioned maps against the single-domain mesh, and the halo
exchange plumbing (face traces) between two gloo ranks.

The kernels need a GPU; what is checked here is everything around them: each
block's local neighbour table (own and ghost records) names exactly the
neighbours of the single-domain mesh, the blocks cover the mesh once, each
side of a cut agrees on the order of the exchanged faces, and an exchange
through torch.distributed (gloo, world size 2) delivers to every ghost face a
local element reads the trace of the element face it stands for.
"""

import ctypes
import os
import socket

import numpy as np
import pytest

from paper_2005_02516_gb300 import esdg
from paper_2005_02516_gb300 import partition as P


def _lib():
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return esdg.load_library()


def _ctx(lib, cfg, part=None):
    h = ctypes.c_void_p()
    if part is None:
        rc = lib.esdg_build_operators(ctypes.byref(cfg), ctypes.byref(h))
    else:
        rc = lib.esdg_build_partition(ctypes.byref(cfg), part[0], part[1], part[2], ctypes.byref(h))
    assert rc == 0, lib.esdg_last_error(None)
    return h


LAYOUTS = [(2, 1), (1, 2), (2, 2), (3, 2), (4, 3)]


@pytest.mark.parametrize("walls", [False, True])
@pytest.mark.parametrize("px,py", LAYOUTS)
def test_partition_maps_reproduce_the_single_domain_mesh(px, py, walls):
    lib = _lib()
    cfg = esdg.make_config(2, 7, 5, warp=0.05, rule="symmetric", walls=walls)
    full = _ctx(lib, cfg)
    F = esdg.partition_layout(lib, full)
    Kg = F["K"]
    xf, yf = np.zeros((Kg, 6)), np.zeros((Kg, 6))
    lib.esdg_get_points(full, esdg.ESDG_POINTS_NODAL, xf.ctypes.data, yf.ctypes.data)
    seen = np.zeros(Kg, dtype=int)
    layouts = []
    for part in range(px * py):
        h = _ctx(lib, cfg, (px, py, part))
        L = esdg.partition_layout(lib, h)
        layouts.append(L)
        assert L["K_global"] == Kg and (L["px"], L["py"], L["part"]) == (px, py, part)
        K, Kp, own, gg = L["K"], P.kpad(L["K"]), L["owned_gid"], L["ghost_gid"]
        assert np.all(np.diff(own) > 0)                      # increasing global order
        seen[own] += 1
        # every face of every local element names the single-domain neighbour
        for k in range(K):
            for f in range(3):
                nb = L["nbr"][k, f]
                en, fn = nb >> 2, nb & 3
                want = F["nbr"][own[k], f]
                if fn == 3:
                    assert en == k and want == 4 * own[k] + 3
                    continue
                assert en < K or (Kp <= en < Kp + L["nghost"])
                gid = own[en] if en < K else gg[en - Kp]
                assert 4 * gid + fn == want
        # ghosts: exactly the non-owned neighbours, sorted by block then element,
        # each owned by the block named
        nb_all = F["nbr"][own].ravel()
        outside = np.unique((nb_all >> 2)[((nb_all & 3) != 3) & ~np.isin(nb_all >> 2, own)])
        assert sorted(gg.tolist()) == outside.tolist()
        keys = list(zip(L["ghost_part"].tolist(), gg.tolist()))
        assert keys == sorted(keys)
        # geometry restricted with the elements
        x, y = np.zeros((K, 6)), np.zeros((K, 6))
        lib.esdg_get_points(h, esdg.ESDG_POINTS_NODAL, x.ctypes.data, y.ctypes.data)
        assert np.array_equal(x, xf[own]) and np.array_equal(y, yf[own])
        lib.esdg_destroy(h)
    assert np.all(seen == 1)                                 # the blocks cover the mesh once
    for L in layouts:
        for g, q in zip(L["ghost_gid"], L["ghost_part"]):
            assert g in set(layouts[q]["owned_gid"].tolist())
    # both sides of every cut agree on the exchanged faces and their order, and
    # every face a block reads from a ghost is received exactly once
    plans = [P.halo_plan(L) for L in layouts]
    for q, plan in enumerate(plans):
        Lq = layouts[q]
        Kp = P.kpad(Lq["K"])
        read = set()
        for k in range(Lq["K"]):
            for f in range(3):
                nb = Lq["nbr"][k, f]
                if (nb & 3) != 3 and (nb >> 2) >= Kp:
                    read.add(4 * ((nb >> 2) - Kp) + (nb & 3))
        got = []
        for r, (send, recv) in plan.items():
            assert q in plans[r]
            sent = [(layouts[q]["owned_gid"][x >> 2], x & 3) for x in send]
            rsend, rrecv = plans[r][q]
            there = [(layouts[r]["ghost_gid"][x >> 2], x & 3) for x in rrecv]
            assert sent == there
            got += recv.tolist()
        assert sorted(got) == sorted(read) and len(got) == len(set(got))
    lib.esdg_destroy(full)


def test_partition_refuses_bad_layouts():
    lib = _lib()
    cfg = esdg.make_config(2, 4, 4)
    h = ctypes.c_void_p()
    for px, py, part in [(0, 1, 0), (2, 2, 4), (2, 2, -1), (5, 1, 0)]:
        assert lib.esdg_build_partition(ctypes.byref(cfg), px, py, part, ctypes.byref(h)) == esdg.ESDG_EINVAL
        assert not h.value


def test_single_block_partition_has_no_ghosts():
    lib = _lib()
    cfg = esdg.make_config(3, 5, 4, warp=0.05)
    h = _ctx(lib, cfg, (1, 1, 0))
    L = esdg.partition_layout(lib, h)
    assert L["nghost"] == 0 and np.array_equal(L["owned_gid"], np.arange(L["K"]))
    assert P.halo_plan(L) == {}
    lib.esdg_destroy(h)


# ---- the exchange between two gloo ranks ----------------------------------------

def _record(gid, nrec):
    # a record block that names its element: (gid, node, component)
    node = np.arange(nrec)[:, None]
    comp = np.arange(4)[None, :]
    return gid * 1000.0 + node * 4.0 + comp


def _rank_main(rank, world, port, px, py, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lib = _lib()
        cfg = esdg.make_config(2, 6, 5, precision="fp64", warp=0.05, rule="symmetric")
        h = _ctx(lib, cfg, (px, py, rank))
        L = esdg.partition_layout(lib, h)
        K, Kp, G = L["K"], P.kpad(L["K"]), L["nghost"]
        Kc, Np, Nq, Nfq = (ctypes.c_int() for _ in range(4))
        lib.esdg_sizes(h, ctypes.byref(Kc), ctypes.byref(Np), ctypes.byref(Nq), ctypes.byref(Nfq), None)
        Nq, Nfp = Nq.value, Nfq.value // 3
        nrec = Nq + Nfq.value
        assert L["trace_bytes"] == 8 * 4 * Nfp
        rec = np.full((Kp + G, nrec, 4), np.nan)
        for k in range(K):
            rec[k] = _record(L["owned_gid"][k], nrec)

        def nodes(f):
            return Nq + f * Nfp + np.arange(Nfp)

        def pack(faces, out):
            tr = np.stack([rec[x >> 2, nodes(x & 3)] for x in faces.numpy()])
            out.view(torch.float64).copy_(torch.from_numpy(tr.ravel()))

        def unpack(buf, faces):
            tr = buf.view(torch.float64).numpy().reshape(-1, Nfp, 4)
            for x, t in zip(faces.numpy(), tr):
                rec[Kp + (x >> 2), nodes(x & 3)] = t

        plan = P.halo_plan(L)
        ex = P.HaloExchange(plan, L["trace_bytes"], pack, unpack, device="cpu")
        P.exchange(ex, P.DistTransport())
        ok, nread = True, 0
        for k in range(K):
            for f in range(3):
                nb = L["nbr"][k, f]
                if (nb & 3) != 3 and (nb >> 2) >= Kp:
                    g, fn = (nb >> 2) - Kp, nb & 3
                    want = _record(L["ghost_gid"][g], nrec)[nodes(fn)]
                    ok = ok and np.array_equal(rec[Kp + g, nodes(fn)], want)
                    nread += 1
        untouched = np.all(np.isnan(rec[K:Kp])) if Kp > K else True
        q.put((rank, bool(ok and nread > 0 and untouched), int(G), ex.bytes_per_exchange()))
        lib.esdg_destroy(h)
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2)])
def test_halo_exchange_between_two_gloo_ranks(px, py):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, px, py, q)) for r in range(2)]
    for p_ in procs:
        p_.start()
    res = [q.get(timeout=180) for _ in procs]
    for p_ in procs:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    assert sorted(r[0] for r in res) == [0, 1]
    assert all(r[1] for r in res), res
