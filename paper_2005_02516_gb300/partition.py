"""Element partition of one solve over several GPUs: the halo plan and the
per-stage exchange of entropy-projected face traces.

A block of the partition (esdg_build_partition) owns the elements of a
rectangle of quads; each element's interface flux (Sec. 2.8) reads the
neighbour's entropy-projected values u~ at the shared face, so after the
projection and after every RK stage each block sends the u~ values at the
nodes of its cut faces (3 (N+1) values a face, stored as 4 per node) and
receives those of its ghosts' faces.  One
exchange per stage is the only communication of the solve; the entropy and
mass diagnostics add one sum over blocks.

This module is host logic only: which local faces each neighbouring block
needs and where received traces go.  Gathering the traces and writing them
into the ghost records runs in the library (esdg_halo_pack, esdg_halo_unpack);
the transport is torch.distributed point-to-point (NCCL between GPUs, gloo on
CPU), or an in-process copy when several blocks share one device.
"""

import numpy as np


def kpad(K):
    """Local element count rounded up to whole batches of 8: the index of the
    first ghost record."""
    return (K + 7) // 8 * 8


def halo_plan(layout):
    """The exchange of one block, from its maps (esdg.partition_layout):
    {peer block: (send, recv)}, both int32 arrays of faces 4 e + f.  send: the
    faces of local elements whose neighbour the peer owns; recv: the faces of
    ghost records (e = ghost index) that local elements read.  Both lists run
    in increasing (global element, face) order, so a face the peer sends is
    the face it stands for here at the same position: the two sides agree on
    the order without talking (each cut face is one face of each side, and
    face adjacency is symmetric)."""
    K = layout["K"]
    Kp = kpad(K)
    nbr = layout["nbr"]
    gp, gg, own = layout["ghost_part"], layout["ghost_gid"], layout["owned_gid"]
    en, fn = nbr >> 2, nbr & 3
    is_ghost = (fn != 3) & (en >= Kp)
    ks, fs = np.nonzero(is_ghost)                 # local element, own face
    g = en[ks, fs] - Kp                            # ghost index and the ghost's face
    gf = fn[ks, fs]
    peer = gp[g]
    plan = {}
    for r in np.unique(peer):
        sel = peer == r
        send_keys = sorted(set(zip(own[ks[sel]].tolist(), fs[sel].tolist(), ks[sel].tolist())))
        recv_keys = sorted(set(zip(gg[g[sel]].tolist(), gf[sel].tolist(), g[sel].tolist())))
        send = np.array([4 * k + f for _, f, k in send_keys], dtype=np.int32)
        recv = np.array([4 * gi + f for _, f, gi in recv_keys], dtype=np.int32)
        assert send.size == recv.size
        plan[int(r)] = (send, recv)
    return plan


class HaloExchange:
    """The per-stage exchange of one block.

    pack(faces, out) gathers the face traces of local faces (4 e + f) into the
    flat byte buffer out; unpack(buf, faces) writes traces into ghost faces
    (Solver.halo_pack / halo_unpack on a GPU).  Buffers are allocated once, on
    `device`.
    """

    def __init__(self, plan, trace_bytes, pack, unpack, device="cuda"):
        import torch
        self.peers = sorted(plan)
        self.trace_bytes = trace_bytes
        self._pack, self._unpack = pack, unpack
        self.send_idx, self.recv_idx, self.send_buf, self.recv_buf = {}, {}, {}, {}
        for r in self.peers:
            send, recv = plan[r]
            self.send_idx[r] = torch.as_tensor(send, dtype=torch.int32, device=device)
            self.recv_idx[r] = torch.as_tensor(recv, dtype=torch.int32, device=device)
            self.send_buf[r] = torch.empty(int(send.size) * trace_bytes, dtype=torch.uint8, device=device)
            self.recv_buf[r] = torch.empty(int(recv.size) * trace_bytes, dtype=torch.uint8, device=device)
        self.primed = False

    def pack(self):
        for r in self.peers:
            if self.send_idx[r].numel():
                self._pack(self.send_idx[r], self.send_buf[r])

    def unpack(self):
        for r in self.peers:
            if self.recv_idx[r].numel():
                self._unpack(self.recv_buf[r], self.recv_idx[r])

    def bytes_per_exchange(self):
        return sum(b.numel() for b in self.send_buf.values())


class DistTransport:
    """Point-to-point through torch.distributed: one send and one receive per
    neighbouring block and exchange, posted together."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, ex):
        import torch.distributed as dist
        ops = []
        for r in ex.peers:
            ops.append(dist.P2POp(dist.isend, ex.send_buf[r], r, group=self.group))
            ops.append(dist.P2POp(dist.irecv, ex.recv_buf[r], r, group=self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


def exchange(ex, transport):
    """One halo exchange of one block: gather, send and receive, scatter."""
    ex.pack()
    transport.exchange(ex)
    ex.unpack()


def exchange_local(exchanges, parts):
    """The halo exchange of several blocks held by one process (every block on
    the same device): each block's receive from r is r's send to it."""
    for ex in exchanges:
        ex.pack()
    for ex, q in zip(exchanges, parts):
        for r in ex.peers:
            ex.recv_buf[r].copy_(exchanges[parts.index(r)].send_buf[q])
    for ex in exchanges:
        ex.unpack()


def step(solver, ex, transport, nsteps, dt, t0=0.0):
    """nsteps LSRK45 steps (Sec. 4) of one block: the first call projects the
    state and exchanges, then each stage is followed by an exchange."""
    if not ex.primed:
        solver.project()
        exchange(ex, transport)
        ex.primed = True
    for n in range(nsteps):
        for s in range(5):
            solver.stage(s, dt, t0 + n * dt)
            exchange(ex, transport)
    return t0 + nsteps * dt


def step_local(solvers, exchanges, parts, nsteps, dt, t0=0.0):
    """The same for several blocks on one device, stage by stage in lockstep
    (each stage launch finishes before the exchange that follows it reads its
    output: all blocks work on one stream)."""
    for s_, ex in zip(solvers, exchanges):
        if not ex.primed:
            s_.project()
    if not all(ex.primed for ex in exchanges):
        exchange_local(exchanges, parts)
        for ex in exchanges:
            ex.primed = True
    for n in range(nsteps):
        for s in range(5):
            for sv in solvers:
                sv.stage(s, dt, t0 + n * dt)
            exchange_local(exchanges, parts)
    return t0 + nsteps * dt


def entropy_sum(solver, t=0.0, group=None):
    """Entropy, mass and entropy rate (Sec. 2.4) of the whole solve: each
    block's FP64 sums, then one all-reduce of the three scalars."""
    import torch
    import torch.distributed as dist
    S, M, R = solver.entropy(t)
    v = torch.tensor([S, M, R], dtype=torch.float64, device="cuda")
    dist.all_reduce(v, group=group)
    return tuple(float(x) for x in v.cpu())
