"""Benchmark: ESDG shallow-water right-hand side + LSRK45 on GB300.

Workload (single large solve): N = 4, 256 x 256 quads -> K = 131072 curved
triangles, smoothed dam break h = 1 + 0.5 tanh(40 (0.3 - r)), u = v = 0,
b = 0.05 exp(-10((x-0.4)^2 + y^2)); FP32 right-hand side with FP64 RK
accumulation.  A step is one LSRK45 step (five stages, each one pass of the
whole per-stage path).  Metric: GDOF-stage/s = K * Np * 5 * steps / time / 1e9.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs an
independent replica (the path has no exchange between separate solves), and
value is the sum over ranks divided by the max time over ranks.
"""

import argparse
import json
import os
import subprocess
import sys
import time

# the CPU baseline is timed single-threaded; set before numpy is imported
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2005_02516_gb300 import workloads as W  # noqa: E402

METRIC = "GDOF-stage/s FP32 vs FP64 per GB300 at stated L2 error; served p50/p99 latency"
UNIT = "GDOF-stage/s"
WL = W.DAM
# DRAM traffic of one stage launch at this workload (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture), per inverse-mass kind, keyed to
# the sha1 of the kernel source it was measured on: reported as null once that
# source changes.
STAGE_TRAFFIC = {"exact": {"source_sha1": "af4faf8528e4b1718a68c0a8481c4b7f877b75ee", "bytes": 426.44e6},
                 "weight_adjusted": {"source_sha1": "af4faf8528e4b1718a68c0a8481c4b7f877b75ee", "bytes": 357.72e6}}
STAGE_SOURCE = os.path.join(ROOT, "paper_2005_02516_gb300", "csrc", "esdg_stage2.cuh")
# Warp instructions per element-stage of the FP32 stage kernel (ncu
# smsp__inst_executed.sum / K on the same kernel at K = 32768), keyed the same
# way: the issue-slot roofline of an issue-bound kernel (one warp instruction
# per cycle per SM sub-partition).  Polling of the bulk-copy barrier adds 0-11%
# that varies from capture to capture (38.0 M and 42.2 M warp instructions
# for the same binary); the lower count is the one used.
STAGE_INSTR = {"exact": {"source_sha1": "af4faf8528e4b1718a68c0a8481c4b7f877b75ee", "per_element_stage": 1044.5}}
# the same for the FP32 DG-SBP stage kernel
SBP_TRAFFIC = {"source_sha1": "bc6a6adb39a7b0f39182f3aa3b747208c033571a", "bytes": 386.1e6}
SBP_SOURCE = os.path.join(ROOT, "paper_2005_02516_gb300", "csrc", "esdg_sbp2.cuh")

# Algorithmic work of one element-stage at degree N: FLOPs (an FMA counts 2) of
# each step of the path, and the bytes each element-stage must move.
def algorithmic_flops(N, Nq, wadg=False, stored_operator=False, composed=False):
    """stored_operator: the metric-averaged skew operator Qskew^{x,k},
    Qskew^{y,k} is read rather than formed each stage (the FP64 path on rules
    with Nq <= 16 stores it), so a pair costs 25 FLOPs instead of 35.
    composed: the inverse mass is read as its products with the shared
    operators, M^-1 Vh^T (lift) and Vh M^-1 Vq^T (projection to the hybrid
    nodes), per element (the FP64 path where Np <= 16 and Nh <= 32), so the
    two inverse-mass products and the separate Vq^T and Vh contractions are
    not done."""
    Np = (N + 1) * (N + 2) // 2
    Nfq = 3 * (N + 1)
    Nh = Nq + Nfq
    pairs = Nq * (Nq - 1) // 2 + Nq * Nfq            # unique non-zero pairs of Q_skew
    flops = 0
    flops += 2 * Nq * Np * 3                          # u_q = Vq u
    flops += 10 * Nq                                  # entropy variables
    if wadg:
        # weight-adjusted inverse through the composed factors A = Vq Vq^T,
        # B = Vh Vq^T, C = Vq Vh^T and the per-node scale w/J
        flops += 3 * Nq + 2 * Nq * Nq * 3 + 4 * Nq    # A (w J v), scale
        flops += 2 * Nh * Nq * 3 + 6 * Nh             # v~ = B z, u~ = u(v~)
    elif composed:
        flops += 3 * Nq + 2 * Nh * Nq * 3 + 6 * Nh        # v~ = (Vh M^-1 Vq^T)(W J v), u~ = u(v~)
    else:
        flops += 2 * Np * Nq * 3 + 3 * Nq + 2 * Np * Np * 3   # J-weighted projection
        flops += 2 * Nh * Np * 3 + 6 * Nh                 # v~ = Vh v_h, u~ = u(v~)
    # flux differencing: 35 flops a unique pair, 10 of them the metric average
    # (four sums, two products and two FMAs) that a stored operator saves
    flops += (25 if stored_operator else 35) * pairs
    flops += 40 * Nfq                                 # interface flux + Lax-Friedrichs
    if wadg:
        flops += 2 * Nq * Nh * 3 + 4 * Nq + 2 * Np * Nq * 3   # C r, scale, Vq^T
    elif composed:
        flops += 2 * Np * Nh * 3                          # (M^-1 Vh^T) r
    else:
        flops += 2 * Np * Nh * 3 + 2 * Np * Np * 3        # lift + inverse mass
    flops += 4 * 3 * Np                               # RK stage (FP64)
    return flops


def algorithmic_bytes(N, Nq, real_bytes=4, wadg=False):
    """Bytes one element-stage of the method must move, whatever the kernel's
    design: the FP64 state and RK residual, the geometry and operators that
    vary per element, and one exchange of face traces between neighbours."""
    Np = (N + 1) * (N + 2) // 2
    Nfq = 3 * (N + 1)
    Nh = Nq + Nfq
    NpP = Np * (Np + 1) // 2
    b = 0
    b += 4 * 3 * Np * 8                 # u read + write, res read + write (FP64)
    b += Nh * 4 * real_bytes            # metrics rxJ sxJ ryJ syJ at the hybrid nodes
    b += Nq * real_bytes                # J at the volume nodes (as w_q J_q)
    b += 0 if wadg else NpP * real_bytes    # packed inverse mass matrix (none when weight-adjusted)
    b += Nfq * 3 * real_bytes           # face normals nxJ, nyJ and sJ
    b += Nh * real_bytes                # bathymetry at the hybrid nodes
    b += 2 * Nfq * 3 * real_bytes       # face traces (h, u, v): own write + neighbour read
    b += Nfq * 4                        # connectivity: the exterior node of each face node (int32)
    return b


def design_bytes(N, Nq, real_bytes=4, wadg=False):
    """Bytes the fused stage kernel itself plans to move per element-stage:
    besides the state, residual and per-element data, it re-reads its own
    entropy-projected record (h, u, v, H at every hybrid node) written by the
    previous stage and writes the next one, reads neighbour traces from those
    records, derives face normals from the metrics and stores one neighbour id
    per face."""
    Np = (N + 1) * (N + 2) // 2
    Nfq = 3 * (N + 1)
    Nh = Nq + Nfq
    NpP = Np * (Np + 1) // 2
    b = 0
    b += 4 * 3 * Np * 8                 # u, res read + write (FP64)
    b += 2 * Nh * 4 * real_bytes        # u~ read (own) + write (next stage)
    b += Nfq * 3 * real_bytes           # neighbour traces (h, u, v)
    b += Nh * 4 * real_bytes            # metrics rxJ sxJ ryJ syJ
    b += Nq * real_bytes                # w_q J_q
    b += 0 if wadg else NpP * real_bytes    # packed inverse mass matrix (none when weight-adjusted)
    b += Nh * real_bytes                # bathymetry at hybrid nodes
    b += 3 * 4                          # neighbour ids
    return b


def sbp_algorithmic(N, Nq, real_bytes=4, stored_operator=False):
    """DG-SBP (Sec. 3) per element-stage: FLOPs and bytes.  Nq nodes (all of
    them rows and columns of the dense skew SBP operator), Nfq = 3(N+1) face
    nodes among them.  stored_operator: the metric-averaged operator is read
    rather than formed (the FP64 path), 25 FLOPs a unique pair instead of 35."""
    Nfq = 3 * (N + 1)
    per_pair = 25 if stored_operator else 35
    flops = per_pair * Nq * (Nq - 1) // 2 + 40 * Nfq + 3 * Nq + 4 * 3 * Nq   # pairs, interface, 1/(wJ), RK
    b = 4 * 3 * Nq * 8                  # u, res read + write (FP64)
    b += 2 * Nq * 4 * real_bytes        # nodal records own read + next write
    b += Nfq * 3 * real_bytes           # neighbour values
    b += Nq * 4 * real_bytes            # metrics
    b += 2 * Nq * real_bytes            # w_q J_q, b
    b += 3 * 4                          # neighbour ids
    return flops, b


def fp64_peak(peaks):
    """FP64 SIMT peak, TFLOP/s: 152 SMs x 2 DFMA per SM per cycle (the unit
    rate ncu states for sm_103) x 2 FLOP x the maximum SM clock."""
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12, "152 SMs x 2 DFMA/cycle x 2 x %.0f MHz" % sm_mhz


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "esdg_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(backend="nccl"):
    """Replica ranks from the torchrun environment (RANK, LOCAL_RANK,
    WORLD_SIZE, MASTER_*).  One process per GPU; the ranks exchange only the
    barrier and the max of their timings."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, world, max_seconds):
    """Whole-job throughput of N replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / max_seconds / 1e9


DENSE = "auto"  # how the FP32 modal path applies the dense operators (--dense)


def make_solver(precision, mass="exact", method="modal", dense=None):
    from paper_2005_02516_gb300.esdg import Solver, ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    s = Solver(WL.N, WL.nx, WL.ny, precision=precision, warp=WL.warp, g=WL.g, cfl=WL.cfl, rule=WL.rule, mass=mass,
               method=method, dense=dense or DENSE)
    xb, yb = s.points(ESDG_POINTS_NODAL)
    xq, yq = s.points(ESDG_POINTS_VOLQ)
    s.init_state(WL.bathymetry(xb, yb), WL.initial(xq, yq))
    return s


def time_steps(s, steps, warmup, world):
    """Device time of `steps` LSRK45 steps (CUDA events on the library's stream)."""
    import torch
    dt = s.dt()
    s.step(warmup, dt, 0.0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    s.step_async(steps, dt, warmup * dt)
    ev1.record(s.stream)
    ev1.synchronize()
    s.check()
    torch.cuda.synchronize()
    barrier(world)
    return ev0.elapsed_time(ev1) / 1e3


def precision_report(s64, nsteps):
    """The FP32 path (FP32 right-hand side, FP64 RK accumulation) against the
    FP64 path after the same nsteps from the same initial state: relative L2
    difference of the modal state and the FP64 entropy diagnostics of both.
    The FP64 path matches the FP64 oracle to relative 1e-12 per step (parity
    tests), so it stands in for the oracle at this size."""
    import numpy as np
    s32 = make_solver("fp32")
    dt = s64.dt()
    s32.step(nsteps, dt, 0.0)
    t = nsteps * dt
    u32, u64 = s32.get_state(), s64.get_state()
    S32, M32, R32 = s32.entropy(t)
    S64, M64, R64 = s64.entropy(t)
    s32.close()
    return {"reference": "FP64 path after the same steps (parity-tested against the FP64 oracle)",
            "steps": nsteps, "state_rel_l2": float(np.linalg.norm(u32 - u64) / np.linalg.norm(u64)),
            "entropy_rel": abs(S32 - S64) / abs(S64), "mass_rel": abs(M32 - M64) / abs(M64),
            "entropy_rate_fp32": R32, "entropy_rate_fp64": R64,
            # the rate itself is tiny early on (LF dissipation only at the front),
            # so its difference is stated absolutely and per unit entropy
            "entropy_rate_abs_diff": abs(R32 - R64), "entropy_rate_diff_per_entropy": abs(R32 - R64) / abs(S64)}


def time_e2e(s, steps, warmup):
    """Same metric through the public API with host buffers: per step, the
    state goes host -> device, one LSRK45 step runs, and the state comes back
    (esdg_step_host: the projection kernel reads the pinned host state over the
    host link and the last stage writes the result back, one call and one
    synchronisation per step)."""
    import torch
    host_in = torch.empty((3, s.K, s.Np), dtype=torch.float64, pin_memory=True).numpy()
    host_out = torch.empty((3, s.K, s.Np), dtype=torch.float64, pin_memory=True).numpy()
    s.get_state(host_in)
    dt = s.dt()
    for _ in range(max(1, warmup)):
        s.step_host(host_in, 1, dt, 0.0, out=host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step_host(host_in, 1, dt, 0.0, out=host_out)
        host_in, host_out = host_out, host_in
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    nbytes = host_in.nbytes
    return el, nbytes


def run_ensemble(n, steps):
    """Batched ensemble: n independent FP32 problems of mixed N and K in one
    persistent launch per stage (graph-replayed), launch shape autotuned."""
    import torch
    from paper_2005_02516_gb300.esdg import Ensemble, Solver, ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    insts = W.ensemble(n=n, steps=steps)
    solvers = []
    for it in insts:
        s = Solver(it.N, it.nx, it.nx, precision="fp32", warp=it.warp, g=it.g, cfl=it.cfl, rule=it.rule)
        xb, yb = s.points(ESDG_POINTS_NODAL)
        xq, yq = s.points(ESDG_POINTS_VOLQ)
        s.init_state(it.bathymetry(xb, yb), it.initial(xq, yq), surface=True)
        solvers.append(s)
    ens = Ensemble(solvers)
    warps, order = ens.autotune()
    ens.step(2)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(solvers[0].stream)
    ens.step_async(steps)
    ev1.record(solvers[0].stream)
    ev1.synchronize()
    el = ev0.elapsed_time(ev1) / 1e3
    ens.step(0)
    units = sum(it.K * it.Np * 5 * steps for it in insts)
    res = {"value": units / el / 1e9, "unit": UNIT, "instances": n, "steps": steps,
           "elements": sum(it.K for it in insts), "seconds": el,
           "degrees": sorted(set(it.N for it in insts)), "autotuned_warps": warps, "autotuned_order": order,
           "launches": 5 * steps}
    ens.close()
    for s in solvers:
        s.close()
    return res


def served_mean_work(samples=20000):
    """Mean DOF-stages of one served request under the served distributions
    (N ~ U{2..5}, K log-uniform in [512, 131072], steps ~ U[100, 2000]), from a
    large sample of the trace generator."""
    tr = W.served_trace(samples, rate=1.0, seed=W.BASE_SEED + 777)
    return float(np.mean([r.K * r.Np * 5 * r.steps for r in tr]))


def run_served(rate, precision, duration_s, budget_gb=64.0, seed=W.BASE_SEED, drain=True, max_wall_s=None):
    """Served form: Poisson arrivals at `rate` per second of solve requests with
    the served distributions (degree 2..5, K log-uniform in [512, 131072],
    steps uniform in [100, 2000], random smooth bathymetry, lake at rest plus a
    bump), for `duration_s` seconds of arrivals.  Each request is built on a host
    thread at its arrival time and submitted to the continuous-batching loop;
    latency is completion minus arrival (host set-up, queueing, admission and
    GPU time included).  The trace depends on the seed only (the rate scales the
    arrival times), so two runs with one seed and rate see the same requests at
    the same times.  drain=False: the server is destroyed max_wall_s after the
    first arrival, ending the requests still queued or running (for a precision
    that cannot keep up with the rate)."""
    import concurrent.futures
    from paper_2005_02516_gb300 import esdg
    n = int(rate * duration_s * 1.5) + 8
    trace = [r for r in W.served_trace(n, rate=rate, seed=seed) if r.t_arrival <= duration_s]
    n = len(trace)
    srv = esdg.Server(hbm_budget_bytes=int(budget_gb * (1 << 30)))
    t0 = time.perf_counter()
    tickets = [None] * n

    def prepare(i):
        req = trace[i]
        p = esdg.Problem(req.N, req.nx, req.nx, precision=precision, warp=req.warp, g=req.g, cfl=req.cfl,
                         rule=req.rule)
        xb, yb = p.points(esdg.ESDG_POINTS_NODAL)
        xq, yq = p.points(esdg.ESDG_POINTS_VOLQ)
        tickets[i] = srv.submit(p, req.bathymetry(xb, yb), req.initial(xq, yq), req.steps, surface=True)

    futs = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=8) as pool:
        for i, req in enumerate(trace):
            delay = req.t_arrival - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            futs.append(pool.submit(prepare, i))
        for f in futs:
            f.result()
    if drain:
        srv.drain(3600.0)
    else:
        left = max_wall_s - (time.perf_counter() - t0)
        if left > 0:
            try:
                srv.drain(left)
            except esdg.EsdgError:
                pass
    wall = time.perf_counter() - t0
    # server clock starts at esdg_server_create, within microseconds of t0
    lat, done_units, last_done = [], 0, 0.0
    for i, req in enumerate(trace):
        state, ts, ta, td = srv.query(tickets[i])
        if state == 2:
            lat.append(td - req.t_arrival)
            done_units += req.K * req.Np * 5 * req.steps
            last_done = max(last_done, td)
        elif drain:
            raise RuntimeError("request %d failed with state %d" % (i, state))
    iters, steps, _, max_active = srv.stats()
    loop_s = srv.timing()
    srv.close()
    lat = np.array(lat) if lat else np.array([np.nan])
    res = {"precision": precision, "rate_per_s": rate, "arrival_window_s": duration_s, "requests": n,
           "completed": int(np.isfinite(lat).sum()), "p50_s": float(np.percentile(lat, 50)),
           "p99_s": float(np.percentile(lat, 99)), "mean_s": float(np.mean(lat)),
           "throughput": done_units / wall / 1e9, "unit": UNIT, "wall_s": wall, "iterations": iters,
           "max_active_in_one_iteration": max_active,
           "loop_seconds": {k: round(v, 3) for k, v in loop_s.items()},
           "drain_after_last_arrival_s": (last_done - trace[-1].t_arrival) if drain and n else None,
           "distributions": "N U{2..5}, K log-uniform [512, 131072], steps U[100, 2000]"}
    return res


def run_volume_ratio(sizes=(16, 32, 50, 100, 150, 200), pairs_gpu=1 << 27, pairs_cpu=4_000_000):
    """The volume-kernel cost comparison of Sec. 5.4: run time of the ESDG
    flux-differencing volume term (Q o F) 1 over that of the traditional DG
    products Q f, with random dense n x n operators (W.volume_ratio_inputs), on
    the GPU (esdg_volume_kernel, FP32 and FP64, CUDA events, about pairs_gpu
    operator entries x elements per launch, operators L2-resident) and on one
    host core (esdg_volume_kernel_host, FP64, about pairs_cpu per call)."""
    import torch
    from paper_2005_02516_gb300 import esdg
    kinds = {"dg": esdg.ESDG_VOLUME_DG, "esdg": esdg.ESDG_VOLUME_ESDG}
    rows = []
    for n in sizes:
        K = max(512, pairs_gpu // (n * n))
        Qx, Qy, u = W.volume_ratio_inputs(n, K)
        row = {"n": n, "K_gpu": K}
        for name, dt in (("gpu_fp32", torch.float32), ("gpu_fp64", torch.float64)):
            dev = [torch.tensor(a, dtype=dt, device="cuda") for a in (Qx, Qy, u)]
            out = torch.empty_like(dev[2])
            t = {}
            for kname, kind in kinds.items():
                for _ in range(2):
                    esdg.volume_kernel(kind, *dev, out=out)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                reps = 5
                ev0.record()
                for _ in range(reps):
                    esdg.volume_kernel(kind, *dev, out=out)
                ev1.record()
                ev1.synchronize()
                t[kname] = ev0.elapsed_time(ev1) / reps / 1e3
            row[name] = {"t_dg_s": t["dg"], "t_esdg_s": t["esdg"], "ratio": t["esdg"] / t["dg"],
                         "esdg_pairs_per_s": K * n * n / t["esdg"]}
            del dev, out
        Kc = max(1, pairs_cpu // (n * n))
        hq = [a[..., :Kc, :] if a.ndim == 3 else a for a in (Qx, Qy, u)]
        hq = [np.ascontiguousarray(a) for a in hq]
        t = {}
        for kname, kind in kinds.items():
            esdg.volume_kernel(kind, *hq)
            t0 = time.perf_counter()
            esdg.volume_kernel(kind, *hq)
            t[kname] = time.perf_counter() - t0
        row["cpu_fp64"] = {"K": Kc, "cores": 1, "t_dg_s": t["dg"], "t_esdg_s": t["esdg"],
                           "ratio": t["esdg"] / t["dg"]}
        rows.append(row)
    return rows


# The paper's V100 FP64 times per LSRK45 step at K = 65536 (optimized kernels;
# Sec. 5.3 table), for the context row.
PAPER_V100_FP64_S_PER_STEP = {1: 0.0221, 2: 0.0316, 3: 0.0515, 4: 0.0627, 5: 0.1585}


GOLDEN_MMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "mms_k8192_n3_1000steps.txt")


def _golden_mms():
    """The stored FP64 oracle values of the manufactured-solution run (sampled
    coefficients of the final state and the oracle's own L2 errors, measured
    with its degree-2N+2 error rule)."""
    idx, val, l2 = [], [], None
    with open(GOLDEN_MMS) as f:
        for line in f:
            if line.startswith("#") or line.startswith("norms"):
                continue
            parts = line.split()
            if parts[0] == "l2err":
                l2 = [float(v) for v in parts[1:4]]
                continue
            idx.append(int(parts[0]))
            val.append(float(parts[1]))
    return np.array(idx), np.array(val), l2


def run_accuracy():
    """The stated-accuracy leg: the manufactured-solution workload (N = 3,
    64 x 64 quads -> K = 8192 curved, forcing, 1000 steps) on the FP32 and the
    FP64 path from the same initial data.  For each: the per-field L2 error
    against the exact solution at the final time (esdg_l2_error, the volume
    rule), its throughput, and the relative difference of the sampled final
    coefficients from the stored FP64 oracle values; plus the FP32-FP64 state
    difference."""
    import torch
    from paper_2005_02516_gb300.esdg import Solver, ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    w = W.MMS
    gidx, gval, gl2 = _golden_mms() if os.path.exists(GOLDEN_MMS) else (None, None, None)
    out = {"workload": w.name, "N": w.N, "K": w.K, "steps": w.steps, "curved": True, "forcing": w.forcing,
           "l2_rule": "the volume rule of the run (collapsed, exact to degree 2N+1)"}
    states = {}
    for prec in ("fp32", "fp64"):
        s = Solver(w.N, w.nx, w.ny, precision=prec, warp=w.warp, g=w.g, cfl=w.cfl, forcing=w.forcing)
        xb, yb = s.points(ESDG_POINTS_NODAL)
        xq, yq = s.points(ESDG_POINTS_VOLQ)
        s.init_state(w.bathymetry(xb, yb), w.initial(xq, yq))
        dt = s.dt()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(s.stream)
        s.step_async(w.steps, dt, 0.0)
        ev1.record(s.stream)
        ev1.synchronize()
        s.check()
        el = ev0.elapsed_time(ev1) / 1e3
        T = w.steps * dt
        err = s.l2_error(w.exact(xq, yq, T))
        u = s.get_state()
        states[prec] = u
        rec = {"l2_error": [float(v) for v in err], "t_final": T,
               "value": s.K * s.Np * 5 * w.steps / el / 1e9, "unit": UNIT, "seconds": el}
        if gidx is not None:
            got = u.ravel()[gidx]
            rec["rel_diff_vs_oracle_samples"] = float(np.linalg.norm(got - gval) / np.linalg.norm(gval))
        out[prec] = rec
        s.close()
    out["fp32_vs_fp64_state_rel_l2"] = float(np.linalg.norm(states["fp32"] - states["fp64"])
                                             / np.linalg.norm(states["fp64"]))
    if gl2 is not None:
        out["oracle_l2_error_degree_2n2_rule"] = gl2
        out["oracle_samples"] = "%d coefficients of the final FP64 oracle state (tests/golden)" % len(gidx)
    return out


def run_sbp(steps, warmup, world, peaks):
    """The DG-SBP scheme of Sec. 3 on the same workload (N = 4, K = 131072
    curved; 22 SBP nodes per element): FP32 right-hand side with FP64 RK and
    the plain FP64 path, time per stage, throughput counted in the modal
    unknowns K Np (same polynomial degree, so comparable with the headline)
    and in its own nodal unknowns K Nq, and the FP32 kernel's HBM roofline."""
    import hashlib
    out = {}
    for prec, st in (("fp32", steps), ("fp64", max(2, steps // 20))):
        s = make_solver(prec, method="sbp")
        el = time_steps(s, st, warmup if prec == "fp32" else 1, world)
        t = el / (5 * st)
        row = {"value": s.K * s.Np * 5 * st / el / 1e9, "unit": UNIT,
               "nodal_gdof_stage_s": s.K * s.Nq * 5 * st / el / 1e9, "ms_per_step": el / st * 1e3, "steps": st,
               "Nq": s.Nq, "device_bytes": s.device_bytes}
        if prec == "fp64":
            pk64, pk64_src = fp64_peak(peaks)
            fl64 = sbp_algorithmic(WL.N, s.Nq, 8, stored_operator=True)[0]
            ach = fl64 * s.K / t / 1e12
            row["roofline"] = {"bound": "alu", "achieved": ach, "peak": pk64, "unit": "TFLOP/s", "frac": ach / pk64,
                               "peak_source": pk64_src, "algorithmic_flops_per_element_stage": fl64,
                               "stored_operator": True}
        if prec == "fp32":
            fl, by = sbp_algorithmic(WL.N, s.Nq, 4)
            traffic = None
            with open(SBP_SOURCE, "rb") as f:
                if SBP_TRAFFIC is not None and hashlib.sha1(f.read()).hexdigest() == SBP_TRAFFIC["source_sha1"]:
                    traffic = SBP_TRAFFIC["bytes"]
            row["roofline"] = {"bound": "hbm", "achieved": by * s.K / t / 1e9, "peak": peaks["hbm_gbs"],
                               "unit": "GB/s", "frac": by * s.K / t / 1e9 / peaks["hbm_gbs"], "traffic": traffic,
                               "algorithmic_bytes_per_element_stage": by, "algorithmic_flops_per_element_stage": fl}
        out[prec] = row
        s.close()
    return out


def run_collapsed(steps, warmup, world, peaks):
    """The same workload (smoothed dam break, N = 4, K = 131072 curved) with the
    collapsed (N+1)^2 = 25-point volume rule instead of the 16-point symmetric
    one (Nh = 40, 675 rather than 360 unique non-zero pairs per element): its
    FP32 throughput and roofline fractions, for comparison with the headline."""
    import dataclasses
    global WL
    saved = WL
    WL = dataclasses.replace(WL, rule="collapsed")
    try:
        s = make_solver("fp32")
        el = time_steps(s, steps, warmup, world)
        t = el / (5 * steps)
        fl, by = algorithmic_flops(WL.N, s.Nq), algorithmic_bytes(WL.N, s.Nq)
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        res = {"volume_rule": "collapsed", "Nq": s.Nq, "value": s.K * s.Np * 5 * steps / el / 1e9, "unit": UNIT,
               "ms_per_step": el / steps * 1e3,
               "hbm": {"achieved": by * s.K / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": by * s.K / t / 1e9 / peaks["hbm_gbs"], "algorithmic_bytes_per_element_stage": by},
               "alu": {"achieved": fl * s.K / t / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                       "frac": fl * s.K / t / 1e12 / fp32_peak, "algorithmic_flops_per_element_stage": fl}}
        s.close()
    finally:
        WL = saved
    return res


def run_dense_other(steps, warmup, world, peaks):
    """The headline workload with the dense contractions (V_q, V_q^T W J, V_h,
    the lift) in the form the headline did not use: on the tensor cores
    (tcgen05, split TF32) when the headline ran them on the FP32 pipes, and the
    other way round.  Throughput and the HBM fraction on the method's bytes."""
    other = "simt" if DENSE == "tensor" else "tensor"
    s = make_solver("fp32", dense=other)
    el = time_steps(s, steps, warmup, world)
    t = el / (5 * steps)
    by = algorithmic_bytes(WL.N, s.Nq)
    res = {"dense": other, "value": s.K * s.Np * 5 * steps / el / 1e9, "unit": UNIT,
           "ms_per_step": el / steps * 1e3, "us_per_stage": t * 1e6,
           "hbm": {"achieved": by * s.K / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                   "frac": by * s.K / t / 1e9 / peaks["hbm_gbs"], "algorithmic_bytes_per_element_stage": by}}
    s.close()
    return res


def run_partition_one_gpu(steps, px=2, py=2):
    """The element partition's machinery on one device: the bench workload split
    into px x py blocks, run as separate contexts with their halos exchanged by
    device copies after every stage (the exchange a multi-GPU run makes over
    NCCL), against the same solve in one context.  Measures the cost of the
    per-stage block launches, gathers and scatters, not communication."""
    import torch
    from paper_2005_02516_gb300 import esdg, partition as P
    parts = list(range(px * py))
    blocks, exs = [], []
    for q in parts:
        s = esdg.Solver(WL.N, WL.nx, WL.ny, precision="fp32", warp=WL.warp, g=WL.g, cfl=WL.cfl, rule=WL.rule,
                        partition=(px, py, q))
        xb, yb = s.points(esdg.ESDG_POINTS_NODAL)
        xq, yq = s.points(esdg.ESDG_POINTS_VOLQ)
        s.init_state(WL.bathymetry(xb, yb), WL.initial(xq, yq))
        L = esdg.partition_layout(s.lib, s.h)
        blocks.append(s)
        exs.append(P.HaloExchange(P.halo_plan(L), L["trace_bytes"], s.halo_pack, s.halo_unpack))
    dt = blocks[0].dt()
    t = P.step_local(blocks, exs, parts, 3, dt, 0.0)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(blocks[0].stream)
    P.step_local(blocks, exs, parts, steps, dt, t)
    ev1.record(blocks[0].stream)
    ev1.synchronize()
    el = ev0.elapsed_time(ev1) / 1e3
    for s in blocks:
        s.check()
    K = sum(s.K for s in blocks)
    halo = sum(ex.bytes_per_exchange() for ex in exs)
    for s in blocks:
        s.close()
    return {"blocks": "%dx%d on one GPU" % (px, py), "value": K * WL.Np * 5 * steps / el / 1e9, "unit": UNIT,
            "ms_per_step": el / steps * 1e3, "halo_bytes_per_stage_all_blocks": halo, "steps": steps}


def run_context(degrees=(1, 2, 3, 4, 5), steps=3):
    """Context row beside the paper's GPU table: K = 65536 affine periodic
    (256 x 128 quads), N = 1..5, the symmetric volume rule (the paper's rule is
    not stated), FP64 and FP32 time per LSRK45 step (CUDA events; the state of
    the smaller degrees fits in L2).  The paper's numbers are for a V100 in
    FP64 with its own quadrature: context, not a like-for-like target."""
    from paper_2005_02516_gb300.esdg import Solver, ESDG_POINTS_NODAL, ESDG_POINTS_VOLQ
    rows = []
    w = W.DAM
    for N in degrees:
        row = {"N": N, "K": 65536, "paper_v100_fp64_s_per_step": PAPER_V100_FP64_S_PER_STEP[N]}
        for prec in ("fp64", "fp32"):
            s = Solver(N, 256, 128, precision=prec, warp=0.0, g=w.g, cfl=w.cfl, rule="symmetric")
            xb, yb = s.points(ESDG_POINTS_NODAL)
            xq, yq = s.points(ESDG_POINTS_VOLQ)
            s.init_state(w.bathymetry(xb, yb), w.initial(xq, yq))
            el = time_steps(s, steps, 1, 1)
            row[prec + "_s_per_step"] = el / steps
            row[prec + "_gdof_stage_s"] = s.K * s.Np * 5 * steps / el / 1e9
            s.close()
        rows.append(row)
    return rows


def _oracle_rhs_loop(o, u, ks, seconds_target, barrier=None):
    """Repeated oracle right-hand sides on the elements ks for about
    seconds_target seconds: (evaluations, seconds)."""
    o.rhs_elements(u, ks)   # warm-up
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    n = 0
    while True:
        o.rhs_elements(u, ks)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds_target:
            return n, el


_CPU_ORACLE = None


def _oracle_worker(i, chunk, seconds_target, barrier, out):
    o, u = _CPU_ORACLE
    ks = np.arange(i * chunk, (i + 1) * chunk)
    out.put(_oracle_rhs_loop(o, u, ks, seconds_target, barrier))


def cpu_baseline(seconds_target=12.0, chunk=2048):
    """The FP64 oracle (as it stands) on the host: right-hand-side evaluations
    on samples of 2048 consecutive elements of the same workload, for about
    `seconds_target` seconds, once on one core and once on every core at the
    same time (one process per core, each on its own 2048 elements; forked,
    so this runs before the process touches the GPU)."""
    global _CPU_ORACLE
    import multiprocessing as mp
    from oracle import Oracle
    o = Oracle(WL.N, WL.nx, WL.ny, ax=WL.warp, ay=WL.warp, g=WL.g, cfl=WL.cfl, rule=WL.rule)
    xb, yb = o.points("nodal")
    o.set_bathymetry(WL.bathymetry(xb, yb))
    xq, yq = o.points("volq")
    u = o.init_state(WL.initial(xq, yq))
    n1, el1 = _oracle_rhs_loop(o, u, np.arange(0, chunk), seconds_target)
    single = chunk * o.Np * n1 / el1 / 1e9
    procs = max(1, min(os.cpu_count() or 1, 64, o.K // chunk))
    _CPU_ORACLE = (o, u)
    ctx = mp.get_context("fork")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(i, chunk, seconds_target, barrier, out)) for i in range(procs)]
    for pr in ps:
        pr.start()
    res = [out.get() for _ in ps]
    for pr in ps:
        pr.join()
    _CPU_ORACLE = None
    parallel = sum(chunk * o.Np * n for n, _ in res) / max(el for _, el in res) / 1e9
    return {"value": parallel, "unit": UNIT, "cores": procs, "kind": "oracle",
            "single_core_value": single,
            "sample": "right-hand-side evaluations of 2048 consecutive elements of the K=131072 N=4 workload "
                      "per core (FP64 numpy oracle, one process per core, %d cores at once, %d-%d evaluations "
                      "each in about %.0f s; one core alone: %d evaluations in %.1f s)"
                      % (procs, min(n for n, _ in res), max(n for n, _ in res), seconds_target, n1, el1)}


def run_reference(args, world, rank):
    """The reference arm: the FP64 oracle (as it stands) on the host, single
    thread, on a bounded sample of the same workload -- 2048 consecutive
    elements, whose right-hand side a stage evaluates (with the entropy
    projection of their neighbours) -- for W warm-up and K timed steps of
    five stages.  Under torchrun only rank 0 runs it."""
    if rank != 0:
        return
    from oracle import Oracle
    o = Oracle(WL.N, WL.nx, WL.ny, ax=WL.warp, ay=WL.warp, g=WL.g, cfl=WL.cfl, rule=WL.rule)
    xb, yb = o.points("nodal")
    o.set_bathymetry(WL.bathymetry(xb, yb))
    xq, yq = o.points("volq")
    u = o.init_state(WL.initial(xq, yq))
    ks = np.arange(0, 2048)
    for _ in range(5 * args.warmup):
        o.rhs_elements(u, ks)
    t0 = time.perf_counter()
    for _ in range(5 * args.steps):
        o.rhs_elements(u, ks)
    el = time.perf_counter() - t0
    value = ks.size * o.Np * 5 * args.steps / el / 1e9
    sample = ("elements 0..2047 of the K=%d N=%d workload, %d steps x 5 right-hand-side evaluations "
              "(FP64 numpy oracle, single thread), %.1f s" % (WL.K, WL.N, args.steps, el))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WL.name, "N": WL.N, "K": WL.K, "Nq": WL.Nq, "volume_rule": WL.rule, "curved": True,
                       "sample_elements": 2048},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def shard_layout(world):
    """Blocks of the element partition for `world` ranks: px x py = world with
    px >= py as close to square as the factors allow."""
    py = int(world ** 0.5)
    while world % py:
        py -= 1
    return world // py, py


def run_shard(args, world, rank, local, peaks):
    """One solve split over the ranks (element partition, one halo exchange of
    the entropy-projected records per RK stage over NCCL): the whole mesh's
    GDOF-stage/s over the slowest rank's time (strong scaling)."""
    import torch
    from paper_2005_02516_gb300 import esdg, partition as P
    px, py = shard_layout(world)
    s = esdg.Solver(WL.N, WL.nx, WL.ny, precision="fp32", warp=WL.warp, g=WL.g, cfl=WL.cfl, rule=WL.rule,
                    partition=(px, py, rank))
    xb, yb = s.points(esdg.ESDG_POINTS_NODAL)
    xq, yq = s.points(esdg.ESDG_POINTS_VOLQ)
    s.init_state(WL.bathymetry(xb, yb), WL.initial(xq, yq))
    L = esdg.partition_layout(s.lib, s.h)
    ex = P.HaloExchange(P.halo_plan(L), L["trace_bytes"], s.halo_pack, s.halo_unpack)
    tr = P.DistTransport()
    dt = s.dt()
    t = P.step(s, ex, tr, args.warmup, dt, 0.0)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    ev0.record(s.stream)
    t = P.step(s, ex, tr, args.steps, dt, t)
    ev1.record(s.stream)
    ev1.synchronize()
    clk = clocks.stop()
    s.check()
    torch.cuda.synchronize()
    barrier(world)
    el = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    S, M, R = P.entropy_sum(s, t) if world > 1 else s.entropy(t)
    K = L["K_global"]
    value = K * s.Np * 5 * args.steps / el / 1e9
    halo = ex.bytes_per_exchange()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WL.name, "N": WL.N, "K": K, "Np": s.Np, "Nq": s.Nq, "volume_rule": WL.rule,
                           "curved": True, "mass": "exact", "method": "modal", "rhs_precision": "fp32",
                           "rk_accumulation": "fp64", "l2": "inputs larger than L2",
                           "parallelism": "element partition %dx%d (one solve)" % (px, py)},
                "shard": {"px": px, "py": py, "local_elements_rank0": L["K"], "ghosts_rank0": L["nghost"],
                          "halo_bytes_per_stage_rank0": halo, "exchanges_per_step": 5,
                          "entropy": S, "mass": M},
                "clocks": clk, "gpu_launches": 5 * args.steps * (1 + len(ex.peers)), "peaks": None}
        print(json.dumps(line))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-volume-ratio", action="store_true", help="skip the DG/ESDG volume-kernel cost comparison")
    ap.add_argument("--no-context", action="store_true", help="skip the K=65536 affine N=1..5 context row")
    ap.add_argument("--fp32-only", action="store_true", help="skip the FP64 and ensemble legs (profiling runs)")
    ap.add_argument("--ensemble", type=int, default=64, help="instances of the batched-ensemble leg (0: skip)")
    ap.add_argument("--ensemble-steps", type=int, default=500)
    ap.add_argument("--served", type=float, default=40.0,
                    help="seconds of Poisson arrivals in the served legs (0: skip)")
    ap.add_argument("--served-load", type=float, default=0.6,
                    help="arrival rate of the served legs as a fraction of the batched FP32 throughput "
                         "over the mean work of a request (the served loop sustains about 0.6: at 0.7 its queue "
                         "grows through the arrival window)")
    ap.add_argument("--dense", default="auto", choices=["auto", "simt", "tensor"],
                    help="dense operators of the FP32 path: FP32 pipes, tensor cores, or the library's choice")
    ap.add_argument("--mass", default="exact", choices=["exact", "weight_adjusted"],
                    help="inverse mass of the timed leg: stored (M_h^k)^-1 (the paper's) or weight-adjusted")
    ap.add_argument("--method", default="modal", choices=["modal", "sbp"],
                    help="scheme of the timed leg: the paper's modal ESDG (Sec. 2) or the DG-SBP scheme (Sec. 3; "
                         "implies --fp32-only --no-e2e)")
    ap.add_argument("--no-sbp", action="store_true", help="skip the DG-SBP comparison leg")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the stated-accuracy leg (manufactured solution, N=3, K=8192, 1000 steps)")
    ap.add_argument("--shard", action="store_true",
                    help="one solve split over the ranks by an element partition (halo exchange per RK stage) "
                         "instead of one replica per rank")
    ap.add_argument("--nx", type=int, default=None,
                    help="grid of nx x nx quads instead of 256 x 256 (small profiling case; not a bench line)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.method == "sbp":   # the side legs belong to the modal headline
        args.fp32_only = args.no_e2e = True
    global WL, DENSE
    DENSE = args.dense
    if args.nx is not None:
        WL = W.scaled(WL, args.nx)
    if args.impl == "reference":
        # CPU work only: the ranks need no process group
        world = int(os.environ.get("WORLD_SIZE", "1"))
        run_reference(args, world, int(os.environ.get("RANK", "0")))
        return
    cb = None
    if int(os.environ.get("WORLD_SIZE", "1")) == 1 and not args.no_cpu_baseline and not args.shard:
        # before any CUDA call: the CPU baseline forks its worker processes
        cb = cpu_baseline()
    world, rank, local = dist_init("nccl")
    import torch
    torch.cuda.set_device(local)
    peaks, peak_kind = load_peaks()
    if args.shard:
        run_shard(args, world, rank, local, peaks)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    s = make_solver("fp32", args.mass, args.method)
    wadg = args.mass == "weight_adjusted"
    sbp_main = args.method == "sbp"
    steps = args.steps
    clocks = ClockSampler(local)
    clocks.start()
    el = time_steps(s, steps, args.warmup, world)
    clk = clocks.stop()
    el_max = max_over_ranks(el, world)
    K, Np, Nq_run = s.K, s.Np, s.Nq
    units = K * Np * 5 * steps
    value = replica_value(units, world, el_max)
    launches = 5 * steps
    t_launch = el / launches
    flops = algorithmic_flops(WL.N, WL.Nq, wadg) * K
    nbytes = algorithmic_bytes(WL.N, WL.Nq, 4, wadg) * K
    if sbp_main:
        fl_s, by_s = sbp_algorithmic(WL.N, s.Nq, 4)
        flops, nbytes = fl_s * K, by_s * K
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12     # TFLOP/s at the maximum SM clock
    alu = flops / t_launch / 1e12
    hbm = nbytes / t_launch / 1e9
    traffic = None
    import hashlib
    rec = (SBP_TRAFFIC if sbp_main else STAGE_TRAFFIC.get(args.mass))
    with open(SBP_SOURCE if sbp_main else STAGE_SOURCE, "rb") as f:
        # captured on the full-size workload only
        if rec is not None and args.nx is None and hashlib.sha1(f.read()).hexdigest() == rec["source_sha1"]:
            traffic = rec["bytes"]
    roof_alu = {"bound": "alu", "achieved": alu, "peak": fp32_peak, "unit": "TFLOP/s", "frac": alu / fp32_peak,
                "traffic": traffic, "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz}
    roof_hbm = {"bound": "hbm", "achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hbm / peaks["hbm_gbs"], "traffic": traffic, "peak_source": peak_kind,
                "algorithmic_bytes_per_element_stage": nbytes / K,
                "design_bytes_per_element_stage": (by_s if sbp_main else design_bytes(WL.N, WL.Nq, 4, wadg))}
    roofline = roof_alu if roof_alu["frac"] >= roof_hbm["frac"] else roof_hbm
    other = roof_hbm if roofline is roof_alu else roof_alu
    # context: the issue-slot roofline (the kernel's own binding limit)
    irec = None if sbp_main else STAGE_INSTR.get(args.mass)
    with open(STAGE_SOURCE, "rb") as f:
        if irec is not None and irec["source_sha1"] == hashlib.sha1(f.read()).hexdigest() and args.dense != "tensor":
            ipe = irec["per_element_stage"]
            issue_peak = 152 * 4 * sm_mhz * 1e6 / 1e9
            other = dict(other)
            other["issue"] = {"bound": "issue", "instructions_per_element_stage": ipe,
                              "achieved": ipe * K / t_launch / 1e9, "peak": issue_peak, "unit": "G warp-instructions/s",
                              "frac": ipe * K / t_launch / 1e9 / issue_peak,
                              "peak_source": "152 SMs x 4 sub-partitions x 1 warp instruction per cycle x %.0f MHz"
                              % sm_mhz}

    # The other inverse-mass kind on the same workload, same steps, for
    # comparison: its throughput, HBM roofline fraction and the relative L2
    # difference of the two FP32 states after the same warm-up + timed steps
    other_mass = None
    if not args.fp32_only and not sbp_main:
        om = "exact" if wadg else "weight_adjusted"
        s2 = make_solver("fp32", om)
        el2 = time_steps(s2, steps, args.warmup, world)
        t2 = el2 / launches
        by2 = algorithmic_bytes(WL.N, WL.Nq, 4, om == "weight_adjusted") * K
        u1, u2 = s.get_state(), s2.get_state()
        other_mass = {"mass": om, "value": K * Np * 5 * steps / el2 / 1e9, "unit": UNIT,
                      "ms_per_step": el2 / steps * 1e3, "steps": steps,
                      "hbm": {"achieved": by2 / t2 / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                              "frac": by2 / t2 / 1e9 / peaks["hbm_gbs"],
                              "algorithmic_bytes_per_element_stage": by2 / K},
                      "device_bytes": s2.device_bytes, "device_bytes_%s" % args.mass: s.device_bytes,
                      "state_rel_l2_between_kinds": float(np.linalg.norm(u2 - u1) / np.linalg.norm(u1))}
        s2.close()
        del s2

    # FP64 right-hand side on the same workload (the plain FP64 path), a few steps
    fp64 = None
    s.close()
    del s
    precision = None
    if not args.fp32_only:
        s64 = make_solver("fp64")
        st64 = max(2, steps // 20)
        el64 = time_steps(s64, st64, 1, world)
        pk64, pk64_src = fp64_peak(peaks)
        Nh = WL.Nq + 3 * (WL.N + 1)
        stored = WL.Nq <= 16 and Nh <= 32            # the FP64 kernel's stored-operator rules
        composed = Np <= 16 and Nh <= 32             # and its stored products with the inverse mass
        fl64 = algorithmic_flops(WL.N, WL.Nq, stored_operator=stored, composed=composed)
        ach64 = fl64 * K * 5 * st64 / el64 / 1e12
        # the same time against the FLOPs of the formulation as written (the
        # metric average formed each stage, the inverse applied after each
        # shared operator)
        fl_form = algorithmic_flops(WL.N, WL.Nq)
        fp64 = {"value": K * Np * 5 * st64 / el64 / 1e9, "unit": UNIT, "ms_per_step": el64 / st64 * 1e3,
                "roofline": {"bound": "alu", "achieved": ach64, "peak": pk64, "unit": "TFLOP/s",
                             "frac": ach64 / pk64, "peak_source": pk64_src,
                             "algorithmic_flops_per_element_stage": fl64, "stored_operator": stored,
                             "composed_inverse_products": composed,
                             "formulation_flops_per_element_stage": fl_form,
                             "frac_on_formulation_flops": fl_form * K * 5 * st64 / el64 / 1e12 / pk64},
                "steps": st64}
        precision = precision_report(s64, 1 + st64)
        s64.close()
        del s64

    sbp = None
    if not args.fp32_only and not args.no_sbp and not sbp_main:
        sbp = run_sbp(steps, args.warmup, world, peaks)

    collapsed = None
    if not args.fp32_only and not sbp_main and args.nx is None:
        collapsed = run_collapsed(steps, args.warmup, world, peaks)

    dense_other = None
    if not args.fp32_only and not sbp_main and args.mass == "exact":
        dense_other = run_dense_other(steps, args.warmup, world, peaks)

    partition_one = None
    if not args.fp32_only and not sbp_main and world == 1:
        partition_one = run_partition_one_gpu(max(10, steps // 5))

    accuracy = None
    if not args.fp32_only and not args.no_accuracy and rank == 0:
        accuracy = run_accuracy()

    volume_ratio = None
    if not args.fp32_only and not args.no_volume_ratio and rank == 0:
        volume_ratio = run_volume_ratio()
    context = None
    if not args.fp32_only and not args.no_context and rank == 0:
        context = run_context()

    ens = None
    if not args.fp32_only and args.ensemble > 0:
        ens = run_ensemble(args.ensemble, args.ensemble_steps)

    served = None
    if not args.fp32_only and args.served > 0 and world == 1:
        # The served distributions unscaled.  The arrival rate is the one the box
        # sustains with FP32 requests: a fraction of the batched throughput over
        # the mean work of a request; FP32 runs that trace for args.served seconds
        # of arrivals and drains.  FP64 then gets the same trace (same requests,
        # same arrival times) for the same window plus a bounded wait: it cannot
        # keep up, so what it completes and its latencies are reported as such.
        mean_work = served_mean_work()
        batched = ens["value"] if ens else 7.0
        rate = args.served_load * batched * 1e9 / mean_work
        s32 = run_served(rate, "fp32", args.served)
        s64 = run_served(rate, "fp64", args.served, drain=False, max_wall_s=args.served + 15.0)
        served = {"mean_work_dof_stages": mean_work, "batched_throughput_used": batched,
                  "load_fraction": args.served_load, "rate_per_s": rate, "fp32": s32, "fp64_same_trace": s64}

    e2e = None
    if not args.no_e2e:
        s = make_solver("fp32")
        e_steps = max(5, steps // 5)
        el_e, nb = time_e2e(s, e_steps, 2)
        el_e = max_over_ranks(el_e, world)
        e2e = {"value": K * Np * 5 * e_steps * world / el_e / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb, "steps": e_steps}
        s.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
                "warmup": args.warmup, "ms_per_step": el_max / steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WL.name if args.nx is None else "%s_nx%d" % (WL.name, args.nx),
                           "N": WL.N, "K": K, "Np": Np, "Nq": Nq_run,
                           "volume_rule": "sbp" if sbp_main else WL.rule, "curved": True,
                           "mass": args.mass, "method": args.method,
                           "dense_contractions": "tensor_cores" if args.dense == "tensor" else "fp32_pipes",
                           "rhs_precision": "fp32", "rk_accumulation": "fp64",
                           "l2": "inputs larger than L2 (state, residual, geometry ~0.5 GB)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": roofline, "roofline_other": other, "other_mass": other_mass, "sbp": sbp,
                "collapsed_rule": collapsed, "dense_other": dense_other, "partition_one_gpu": partition_one,
                "fp64": fp64, "precision": precision, "accuracy": accuracy, "volume_ratio": volume_ratio, "context": context, "ensemble": ens, "served": served, "e2e": e2e, "cpu_baseline": cb, "clocks": clk,
                "gpu_launches": launches, "peaks": peak_kind}
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
