"""The multi-rank plumbing of bench.py on CPU ranks (gloo, world size 2):
replicas join a barrier, agree on the maximum of their timings, and the
whole-job value counts every rank's units over the slowest rank's time."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init("gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + rank, w, device="cpu")
    out.put((rank, t, bench.replica_value(1e9, w, t)))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_replica_ranks_agree_on_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, v in res:
        assert t == 2.0              # the slowest rank's time
        assert abs(v - 1.0) < 1e-12  # 2 ranks x 1e9 units / 2 s / 1e9


def test_accuracy_leg_reads_the_stored_oracle_values():
    """The bench's stated-accuracy leg compares the sampled final coefficients
    with the stored FP64 oracle run (tests/golden): the reader finds the 4000
    samples, distinct indices, and the oracle's three L2 errors."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    idx, val, l2 = bench._golden_mms()
    assert len(idx) == len(val) == 4000 and len(set(idx.tolist())) == 4000
    assert l2 is not None and len(l2) == 3 and all(0 < e < 1e-6 for e in l2)


def test_shard_layout_factors_the_ranks():
    import bench
    for world, want in [(1, (1, 1)), (2, (2, 1)), (3, (3, 1)), (4, (2, 2)), (6, (3, 2)), (8, (4, 2)), (16, (4, 4))]:
        px, py = bench.shard_layout(world)
        assert (px, py) == want and px * py == world
