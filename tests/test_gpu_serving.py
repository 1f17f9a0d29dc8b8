"""Served form: the continuous-batching request loop (esdg_server_*).

Requests of mixed degree, size, precision and step count arrive while others
run; each finished state must equal the same problem run alone through the
single-problem path: FP64 requests to relative 1e-12; FP32 requests to
relative 1e-6 (the ensemble kernel that carries degree-5 members is a
separate compilation of the same arithmetic, whose FP32 roundings may differ
in a few operations; the FP32 accuracy target is 1e-5).  Requests overlap on
the device (continuous batching, not a queue), served results match the FP64
oracle directly, admission respects the HBM budget, a request larger than
the whole budget is refused, and destroying the server ends running requests
promptly.
"""

import time

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


def _prepare(req, precision):
    from paper_2005_02516_gb300 import esdg
    p = esdg.Problem(req.N, req.nx, req.nx, precision=precision, warp=req.warp, g=req.g, cfl=req.cfl,
                     rule=req.rule)
    xb, yb = p.points(esdg.ESDG_POINTS_NODAL)
    xq, yq = p.points(esdg.ESDG_POINTS_VOLQ)
    return p, req.bathymetry(xb, yb), req.initial(xq, yq)


def _alone(req, precision, b, q):
    from paper_2005_02516_gb300 import esdg
    s = esdg.Solver(req.N, req.nx, req.nx, precision=precision, warp=req.warp, g=req.g, cfl=req.cfl,
                    rule=req.rule)
    s.init_state(b, q, surface=True)
    s.step(req.steps)
    u = s.get_state()
    s.close()
    return u


@pytest.mark.parametrize("rules", ["symmetric", "mixed"])
def test_served_results_equal_alone(rules):
    import dataclasses
    from paper_2005_02516_gb300 import esdg
    trace = W.served_trace(8, rate=50.0, seed=W.BASE_SEED + 5, k_range=(32, 800), steps_range=(3, 45))
    if rules == "mixed":   # FP32 requests of both rules: one ensemble per rule
        trace = [dataclasses.replace(r, rule="collapsed" if i % 2 else "symmetric") for i, r in enumerate(trace)]
    precisions = ["fp32", "fp32", "fp64", "fp32", "fp64", "fp32", "fp32", "fp64"]
    srv = esdg.Server(hbm_budget_bytes=4 << 30)
    t0 = time.perf_counter()
    tickets, inputs = [], []
    for req, prec in zip(trace, precisions):
        while time.perf_counter() - t0 < req.t_arrival:
            time.sleep(0.001)
        p, b, q = _prepare(req, prec)
        tickets.append(srv.submit(p, b, q, req.steps, surface=True))
        inputs.append((b, q))
    srv.drain(300.0)
    iters, steps, inuse, _ = srv.stats()
    assert inuse == 0 and iters > 0
    tm = srv.timing()  # the worker's time by phase: all non-negative, and it waited on the GPU
    assert set(tm) == {"admit", "rebuild", "launch", "wait", "retire"}
    assert all(v >= 0.0 for v in tm.values()) and tm["wait"] > 0.0
    for tk, req, prec, (b, q) in zip(tickets, trace, precisions, inputs):
        state, ts, ta, td = srv.query(tk)
        assert state == 2 and ts <= ta <= td
        want = _alone(req, prec, b, q)
        got = srv.result(tk)
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
    srv.close()


def test_admission_respects_the_budget():
    from paper_2005_02516_gb300 import esdg
    trace = W.served_trace(5, rate=1000.0, seed=W.BASE_SEED + 6, k_range=(200, 200), steps_range=(30, 30),
                           degrees=(3,))
    probe, _, _ = _prepare(trace[0], "fp32")
    per = probe.device_bytes + 512
    probe.close()
    srv = esdg.Server(hbm_budget_bytes=2 * per + per // 2)   # room for two at a time
    tickets = []
    for req in trace:
        p, b, q = _prepare(req, "fp32")
        tickets.append(srv.submit(p, b, q, req.steps, surface=True))
    srv.drain(300.0)
    spans = []
    for tk in tickets:
        state, ts, ta, td = srv.query(tk)
        assert state == 2
        spans.append((ta, td))
    for ta, _ in spans:   # never more than two running at once
        running = sum(1 for a, d in spans if a <= ta < d)
        assert running <= 2
    srv.close()


def test_request_larger_than_budget_is_refused():
    from paper_2005_02516_gb300 import esdg
    req = W.served_trace(1, rate=1.0, seed=1, k_range=(800, 800), steps_range=(5, 5), degrees=(4,))[0]
    srv = esdg.Server(hbm_budget_bytes=1 << 20)
    p, b, q = _prepare(req, "fp32")
    with pytest.raises(esdg.EsdgError) as ei:
        srv.submit(p, b, q, req.steps, surface=True)
    assert ei.value.code == esdg.ESDG_EBUSY
    p.close()
    srv.close()


def test_failing_request_does_not_disturb_the_others():
    """A request whose depth is negative somewhere fails with
    ESDG_ENONPOSITIVE or ESDG_ENONFINITE (the device status word of its own
    context) while the
    requests batched with it, FP32 in the same ensemble launch and FP64 beside
    it, finish with the same states as alone."""
    from paper_2005_02516_gb300 import esdg
    trace = W.served_trace(6, rate=1000.0, seed=W.BASE_SEED + 7, k_range=(60, 300), steps_range=(8, 12),
                           degrees=(2, 3))
    precisions = ["fp32", "fp32", "fp64", "fp32", "fp64", "fp32"]
    bad = {1, 4}
    srv = esdg.Server(hbm_budget_bytes=4 << 30)
    tickets, inputs = [], []
    for i, (req, prec) in enumerate(zip(trace, precisions)):
        p, b, q = _prepare(req, prec)
        if i in bad:
            q = q.copy()
            q[0, 0, 0] = -1.0          # a dry point with negative depth
        tickets.append(srv.submit(p, b, q, req.steps, surface=False if i in bad else True))
        inputs.append((b, q))
    srv.drain(300.0)
    for i, (tk, req, prec, (b, q)) in enumerate(zip(tickets, trace, precisions, inputs)):
        state = srv.query(tk)[0]
        if i in bad:
            # the first stage flags the depth (and, from the division by it,
            # non-finite values): either status reports the failed request
            assert state in (esdg.ESDG_ENONPOSITIVE, esdg.ESDG_ENONFINITE)
            continue
        assert state == 2
        want = _alone(req, prec, b, q)
        got = srv.result(tk)
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
    assert srv.stats()[2] == 0        # every request's device memory returned
    srv.close()


def test_served_fp64_requests_of_any_configuration():
    """FP64 requests run through their own contexts: a forced manufactured
    solution (its simulated time carried across the served iterations), a
    DG-SBP problem and a weight-adjusted one finish with the states of the
    same problems run alone (relative 1e-12)."""
    from paper_2005_02516_gb300 import esdg
    mms, dam = W.scaled(W.MMS, 6, 5, N=3), W.scaled(W.DAM, 6, 6, N=3)
    cases = [(mms, dict(forcing="mms_sine", rule="collapsed"), False, 33),
             (dam, dict(method="sbp"), False, 17),
             (dam, dict(mass="weight_adjusted", rule="symmetric"), False, 25)]
    srv = esdg.Server(hbm_budget_bytes=2 << 30)
    tickets, wants = [], []
    for w, kw, surface, steps in cases:
        common = dict(precision="fp64", warp=w.warp, g=w.g, cfl=w.cfl, **kw)
        p = esdg.Problem(w.N, w.nx, w.ny, **common)
        xb, yb = p.points(esdg.ESDG_POINTS_NODAL)
        xq, yq = p.points(esdg.ESDG_POINTS_VOLQ)
        b, q = w.bathymetry(xb, yb), w.initial(xq, yq)
        tickets.append(srv.submit(p, b, q, steps, surface=surface))
        s = esdg.Solver(w.N, w.nx, w.ny, **common)
        s.init_state(b, q, surface=surface)
        s.step(steps)
        wants.append(s.get_state())
        s.close()
    srv.drain(300.0)
    for tk, want in zip(tickets, wants):
        assert srv.query(tk)[0] == 2
        got = srv.result(tk)
        assert np.linalg.norm(got - want) <= 1e-12 * np.linalg.norm(want)
    srv.close()


def test_served_results_match_the_oracle():
    """Served requests against the FP64 oracle directly: FP64 requests at
    relative 1e-12, FP32 ones (25 steps: 20 in an ensemble launch, the last 5
    on their own stage kernels) at relative 1e-5 in the L2 and the max norm."""
    from oracle import Oracle
    from paper_2005_02516_gb300 import esdg
    from _bounds import check_state
    trace = W.served_trace(4, rate=1000.0, seed=W.BASE_SEED + 8, k_range=(32, 80), steps_range=(25, 25),
                           degrees=(2, 3))
    precisions = ["fp32", "fp64", "fp32", "fp64"]
    srv = esdg.Server(hbm_budget_bytes=4 << 30)
    tickets = []
    for req, prec in zip(trace, precisions):
        p, b, q = _prepare(req, prec)
        tickets.append(srv.submit(p, b, q, req.steps, surface=True))
    srv.drain(300.0)
    for tk, req, prec in zip(tickets, trace, precisions):
        assert srv.query(tk)[0] == 2
        o = Oracle(req.N, req.nx, req.nx, ax=req.warp, ay=req.warp, g=req.g, cfl=req.cfl, rule=req.rule)
        xo, yo = o.points("nodal")
        o.set_bathymetry(req.bathymetry(xo, yo))
        xq, yq = o.points("volq")
        u0 = o.init_state(req.initial(xq, yq), surface=True)
        want, _ = o.run(u0, req.steps)
        got = srv.result(tk)
        check_state(got, want, 1e-12 if prec == "fp64" else 1e-5)
    srv.close()


def test_destroy_ends_running_requests():
    """esdg_server_destroy drops queued requests and ends running ones after
    their current iteration (at most 20 steps), so it returns promptly even
    with long FP64 requests on the device."""
    from paper_2005_02516_gb300 import esdg
    trace = W.served_trace(3, rate=1000.0, seed=W.BASE_SEED + 9, k_range=(8192, 8192), steps_range=(5000, 5000),
                           degrees=(4,))
    srv = esdg.Server(hbm_budget_bytes=4 << 30, max_active=1)
    tickets = []
    for req in trace:
        p, b, q = _prepare(req, "fp64")
        tickets.append(srv.submit(p, b, q, req.steps, surface=True))
    time.sleep(1.0)
    t0 = time.perf_counter()
    srv.lib.esdg_server_destroy(srv.h)   # the C ABI call itself, timed
    srv.h = None
    # one request runs (about 10 s of FP64 work in all); ending it after its
    # current 20-step iteration takes a fraction of a second
    assert time.perf_counter() - t0 < 3.0


def test_requests_overlap_on_the_device():
    """Continuous batching, not a queue: a burst of FP32 and FP64 requests is
    admitted while others run, several are advanced by one iteration, and each
    result still equals the same problem run alone."""
    from paper_2005_02516_gb300 import esdg
    trace = W.served_trace(6, rate=1000.0, seed=W.BASE_SEED + 10, k_range=(512, 2048), steps_range=(60, 200),
                           degrees=(2, 3, 4))
    precisions = ["fp32", "fp64", "fp32", "fp32", "fp64", "fp32"]
    srv = esdg.Server(hbm_budget_bytes=4 << 30)
    tickets, inputs = [], []
    for req, prec in zip(trace, precisions):
        p, b, q = _prepare(req, prec)
        tickets.append(srv.submit(p, b, q, req.steps, surface=True))
        inputs.append((b, q))
    srv.drain(300.0)
    _, _, _, max_active = srv.stats()
    assert max_active >= 2
    spans = [srv.query(tk)[2:] for tk in tickets]
    # some request was admitted while another was still running
    assert any(a2 < d1 and a1 < d2 for i, (a1, d1) in enumerate(spans) for j, (a2, d2) in enumerate(spans)
               if i != j)
    for tk, req, prec, (b, q) in zip(tickets, trace, precisions, inputs):
        want = _alone(req, prec, b, q)
        tol = 1e-12 if prec == "fp64" else 1e-6
        assert np.linalg.norm(srv.result(tk) - want) <= tol * np.linalg.norm(want)
    srv.close()
