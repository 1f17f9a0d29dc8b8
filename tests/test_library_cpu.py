"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/esdg.h declares, and its host-side set-up (argument validation, mesh
and point construction, which touch no GPU) agrees with the oracle's
conventions.  No compute call runs here."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2005_02516_gb300 import esdg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    if not os.path.exists(esdg.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return esdg.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "esdg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(esdg_\w+)\s*\(", src, re.M)))


def test_header_declarations_match_binding():
    assert _declared() == sorted(esdg.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _lib()
    for name in _declared():
        assert hasattr(lib, name), name


def _cfg(**kw):
    c = esdg.Config()
    c.N, c.nx, c.ny = kw.get("N", 2), kw.get("nx", 4), kw.get("ny", 4)
    c.precision = kw.get("precision", esdg.ESDG_FP64)
    c.x0, c.x1, c.y0, c.y1 = -1.0, 1.0, -1.0, 1.0
    c.warp_ax = c.warp_ay = kw.get("warp", 0.0)
    c.g, c.cfl = kw.get("g", 1.0), 0.25
    c.lax_friedrichs, c.forcing = 1, 0
    c.volume_rule = kw.get("rule", esdg.ESDG_RULE_COLLAPSED)
    c.boundary = kw.get("boundary", esdg.ESDG_BOUNDARY_PERIODIC)
    c.mass = kw.get("mass", esdg.ESDG_MASS_EXACT)
    c.method = kw.get("method", esdg.ESDG_METHOD_MODAL)
    c.dense = kw.get("dense", esdg.ESDG_DENSE_AUTO)
    return c


def _build(**kw):
    lib = _lib()
    h = ctypes.c_void_p()
    rc = lib.esdg_build_operators(ctypes.byref(_cfg(**kw)), ctypes.byref(h))
    return lib, rc, h


@pytest.mark.parametrize("bad", [dict(N=0), dict(N=6), dict(nx=2), dict(ny=1), dict(g=0.0), dict(precision=7),
                                 dict(rule=2), dict(rule=-1), dict(boundary=2), dict(mass=2), dict(mass=-1),
                                 dict(method=2), dict(method=1, boundary=1), dict(method=1, mass=1)])
def test_build_rejects_bad_config(bad):
    lib, rc, h = _build(**bad)
    assert rc == esdg.ESDG_EINVAL
    assert not h.value
    assert len(lib.esdg_last_error(None)) > 0


def test_build_rejects_folding_warp():
    # an amplitude large enough to fold elements makes J <= 0 somewhere
    lib, rc, h = _build(N=3, nx=8, ny=8, warp=2.0)
    assert rc == esdg.ESDG_EINVAL
    assert b"Jacobian" in lib.esdg_last_error(None)


def test_calls_out_of_order_are_refused():
    lib, rc, h = _build()
    assert rc == 0
    u = np.zeros((3, 32, 6))
    assert lib.esdg_set_state(h, u.ctypes.data, 0) == esdg.ESDG_ESTATE
    assert lib.esdg_step(h, 1, 0.01, None) == esdg.ESDG_ESTATE
    err = (ctypes.c_double * 3)()
    assert lib.esdg_l2_error(h, u.ctypes.data, err) == esdg.ESDG_ESTATE
    assert lib.esdg_l2_error(None, u.ctypes.data, err) == esdg.ESDG_EINVAL
    lib.esdg_destroy(h)


@pytest.mark.parametrize("N,warp,rule", [(1, 0.0, "collapsed"), (2, 0.05, "collapsed"), (4, 0.05, "collapsed"),
                                         (5, 0.0, "collapsed"), (1, 0.05, "symmetric"), (2, 0.0, "symmetric"),
                                         (3, 0.05, "symmetric"), (4, 0.05, "symmetric"), (5, 0.05, "symmetric")])
def test_points_and_sizes_match_oracle_conventions(N, warp, rule):
    # For the symmetric rule this compares two independent constructions (the
    # host builder's and the oracle's Newton solves of the moment equations).
    from oracle import Oracle
    code = esdg.ESDG_RULE_SYMMETRIC if rule == "symmetric" else esdg.ESDG_RULE_COLLAPSED
    lib, rc, h = _build(N=N, nx=5, ny=3, warp=warp, rule=code)
    assert rc == 0
    K, Np, Nq, Nfq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb = ctypes.c_size_t()
    assert lib.esdg_sizes(h, ctypes.byref(K), ctypes.byref(Np), ctypes.byref(Nq), ctypes.byref(Nfq),
                          ctypes.byref(nb)) == 0
    o = Oracle(N, 5, 3, ax=warp, ay=warp, rule=rule)
    assert (K.value, Np.value, Nq.value, Nfq.value) == (o.K, o.Np, o.Nq, o.Nfq)
    assert nb.value > 0
    for kind, okind, n in [(esdg.ESDG_POINTS_NODAL, "nodal", Np.value), (esdg.ESDG_POINTS_VOLQ, "volq", Nq.value),
                           (esdg.ESDG_POINTS_FACEQ, "faceq", Nfq.value)]:
        x, y = np.zeros((K.value, n)), np.zeros((K.value, n))
        assert lib.esdg_get_points(h, kind, x.ctypes.data, y.ctypes.data) == 0
        xo, yo = o.points(okind)
        # quadrature points may be listed in another order: compare as sets per element
        key = lambda a, b: np.lexsort((np.round(b, 9), np.round(a, 9)))  # noqa: E731
        for e in range(K.value):
            i, j = key(x[e], y[e]), key(xo[e], yo[e])
            assert np.abs(x[e, i] - xo[e, j]).max() < 1e-13
            assert np.abs(y[e, i] - yo[e, j]).max() < 1e-13
    dt = ctypes.c_double()
    assert lib.esdg_dt(h, ctypes.byref(dt)) == 0
    assert abs(dt.value - o.dt()) < 1e-15
    lib.esdg_destroy(h)


@pytest.mark.parametrize("N,rule", [(2, "collapsed"), (4, "symmetric")])
def test_walled_mesh_points_match_oracle(N, rule):
    # walls change the connectivity only: the same curved points and the same
    # boundary nodes as the oracle's walled mesh
    from oracle import Oracle
    code = esdg.ESDG_RULE_SYMMETRIC if rule == "symmetric" else esdg.ESDG_RULE_COLLAPSED
    lib, rc, h = _build(N=N, nx=5, ny=4, warp=0.05, rule=code, boundary=esdg.ESDG_BOUNDARY_WALLS)
    assert rc == 0
    o = Oracle(N, 5, 4, ax=0.05, ay=0.05, rule=rule, walls=True)
    x, y = np.zeros((o.K, o.Nfq)), np.zeros((o.K, o.Nfq))
    assert lib.esdg_get_points(h, esdg.ESDG_POINTS_FACEQ, x.ctypes.data, y.ctypes.data) == 0
    xo, yo = o.points("faceq")
    assert np.abs(x - xo).max() < 1e-13 and np.abs(y - yo).max() < 1e-13
    lib.esdg_destroy(h)


@pytest.mark.parametrize("precision", [esdg.ESDG_FP64, esdg.ESDG_FP32])
@pytest.mark.parametrize("rule", [esdg.ESDG_RULE_COLLAPSED, esdg.ESDG_RULE_SYMMETRIC])
def test_weight_adjusted_mass_stores_no_inverses(rule, precision):
    """The weight-adjusted inverse keeps no per-element matrix on the device:
    the footprint drops by the stored inverses, K Np(Np+1)/2 values of the
    RHS precision, less the few KB that the FP32 kernel's composed shared
    operators add (both with the dense operators on the FP32 pipes).  The
    FP64 path with the stored inverse also keeps the inverse's products
    M^-1 Vh^T and Vh M^-1 Vq^T per element where its lane mapping covers them
    (Np <= 16, Nh <= 32: here the 16-point rule), in its padded lane layout
    of ((Nh + 1) / 2 + Nq) 32 doubles."""
    sizes = {}
    for mass in (esdg.ESDG_MASS_EXACT, esdg.ESDG_MASS_WEIGHT_ADJUSTED):
        lib, rc, h = _build(N=4, nx=16, ny=16, warp=0.05, rule=rule, precision=precision, mass=mass,
                            dense=esdg.ESDG_DENSE_SIMT)
        assert rc == 0
        K, Np, Nq, Nfq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nb = ctypes.c_size_t()
        assert lib.esdg_sizes(h, ctypes.byref(K), ctypes.byref(Np), ctypes.byref(Nq), ctypes.byref(Nfq),
                              ctypes.byref(nb)) == 0
        sizes[mass] = (K.value, Np.value, Nq.value, Nfq.value, nb.value)
        lib.esdg_destroy(h)
    K, Np, Nq, Nfq, exact = sizes[esdg.ESDG_MASS_EXACT]
    wadg = sizes[esdg.ESDG_MASS_WEIGHT_ADJUSTED][4]
    rs = 4 if precision == esdg.ESDG_FP32 else 8
    stored = K * Np * (Np + 1) // 2 * rs
    Nh = Nq + Nfq
    if precision == esdg.ESDG_FP64 and Np <= 16 and Nh <= 32:
        assert rule == esdg.ESDG_RULE_SYMMETRIC
        stored += K * ((Nh + 1) // 2 + Nq) * 32 * 8
    assert stored - 16384 <= exact - wadg <= stored + 16384


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_sbp_rule_points_match_oracle(N):
    """The host builder's SBP rule (its own Levenberg-Marquardt solve) gives
    the oracle's nodes in the oracle's order, on a curved mesh."""
    from oracle.sbp import SBPOracle
    lib, rc, h = _build(N=N, nx=5, ny=3, warp=0.05, method=esdg.ESDG_METHOD_SBP)
    assert rc == 0
    o = SBPOracle(N, 5, 3, ax=0.05, ay=0.05)
    K, Nq = ctypes.c_int(), ctypes.c_int()
    assert lib.esdg_sizes(h, ctypes.byref(K), None, ctypes.byref(Nq), None, None) == 0
    assert (K.value, Nq.value) == (o.K, o.Nq)
    x, y = np.zeros((o.K, o.Nq)), np.zeros((o.K, o.Nq))
    assert lib.esdg_get_points(h, esdg.ESDG_POINTS_VOLQ, x.ctypes.data, y.ctypes.data) == 0
    xo, yo = o.points("volq")
    assert np.abs(x - xo).max() < 1e-13 and np.abs(y - yo).max() < 1e-13
    lib.esdg_destroy(h)


def _replay_fp64_pieces(Nq, Nh):
    """The larger rules' schedule (Smem::PIECES): the non-zero pairs
    row-major (volume rows x Nh columns, face rows x Nq columns) in 32 pieces
    of PL; every pair once, at most PR filed rows a piece, and each row's
    pieces inside the lane range its owner reads."""
    NPAIR = Nq * Nh + (Nh - Nq) * Nq
    PL = (NPAIR + 31) // 32
    PR = (PL + Nq - 2) // Nq + 1
    seen, filed = {}, {}
    for lane in range(32):
        p0, p1 = lane * PL, min(lane * PL + PL, NPAIR)
        pp = p0 if p0 < p1 else 0
        if pp < Nq * Nh:
            r, m, ln = pp // Nh, pp % Nh, Nh
        else:
            q = pp - Nq * Nh
            r, m, ln = Nq + q // Nq, q % Nq, Nq
        slot = 0
        for it in range(PL):
            if p0 + it < p1:
                assert r < Nh and m < ln
                seen[(r, m)] = seen.get((r, m), 0) + 1
                m += 1
                if m == ln or p0 + it + 1 == p1:
                    filed.setdefault(r, []).append(lane)
                    slot += 1
                    assert slot <= PR
                    if m == ln and r + 1 < Nh:
                        r, m = r + 1, 0
                        ln = Nh if r < Nq else Nq
    assert seen == {(l, m): 1 for l in range(Nh) for m in range(Nh if l < Nq else Nq)}
    for l in range(Nh):
        start = l * Nh if l < Nq else Nq * Nh + (l - Nq) * Nq
        ln = Nh if l < Nq else Nq
        k0, k1 = start // PL, (start + ln - 1) // PL
        assert set(filed[l]) <= set(range(k0, k1 + 1)) and k1 < 32


def _replay_fp64_diagonals(Nq, Nh):
    """The schedule of esdg_kernels.cuh, k_stage, for Nq <= 16 and Nh <= 32:
    lanes j = lane & 15 of half-warp hf evaluate the pair (j, j + d mod Nq)
    on the volume-volume diagonals (half 0: d = 1..SVV0, half 1: the rest,
    d = Nq / 2 taken by j < Nq / 2 only) and (j, Nq + (j + t) mod L) on the
    volume-face diagonals (L = max(Nq, Nfq), half 0: t < SVF0); each step
    every row takes the transposed term of the lane d (or t) places before it
    in its half.  Returns the evaluated pairs and the delivered terms."""
    V, F = Nq, Nh - Nq
    L = max(V, F)
    assert L <= 16
    SVV = V // 2
    SVV0 = (SVV + 1) // 2
    SVF0 = (L + 1) // 2
    evaluated, delivered = {}, {}
    for hf in range(2):
        for k in range(SVV0):
            d = 1 + k if hf == 0 else SVV0 + 1 + k
            step = d <= SVV
            sent = {}
            for j in range(16):
                act = j < V and step and not (2 * d == V and j >= V // 2)
                m = (j + d) % V if j < V else None
                if act:
                    evaluated[frozenset((j, m))] = evaluated.get(frozenset((j, m)), 0) + 1
                    sent[j] = (j, m)          # the transposed term of pair (j, m) for row m
            for j in range(16):
                src = (j - d) % V if j < V else (j - d) % V
                if j < V and step and src in sent:
                    pl, pm = sent[src]
                    assert pm == j, "a transposed term reached the wrong row"
                    delivered[(pl, pm)] = delivered.get((pl, pm), 0) + 1
        for k in range(SVF0):
            t = k if hf == 0 else SVF0 + k
            step = t < L
            sent = {}
            for j in range(16):
                f = (j + t) % L
                act = j < V and step and f < F
                if act:
                    key = (j, V + f)
                    evaluated[frozenset(key)] = evaluated.get(frozenset(key), 0) + 1
                    sent[j] = key
            for j in range(16):
                src = (j - t) % L
                if step and j < F and src in sent:
                    pl, pm = sent[src]
                    assert pm == V + j, "a transposed term reached the wrong face row"
                    delivered[(pl, pm)] = delivered.get((pl, pm), 0) + 1
    return evaluated, delivered


@pytest.mark.parametrize("rule", ["collapsed", "symmetric"])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_fp64_kernel_pair_assignment_covers_each_pair_once(N, rule):
    """The FP64 stage kernel's lane schedule of the pair loop, replayed on the
    host: with Nq <= 16 and Nh <= 32 every non-zero pair of Q_skew (volume x
    volume, volume x face; the face-face block is zero) is evaluated exactly
    once and its transposed term reaches its other row exactly once; the
    larger rules' 32-piece schedule covers every ordered non-zero pair once."""
    Nq = {1: 3, 2: 6, 3: 12, 4: 16, 5: 25}[N] if rule == "symmetric" else (N + 1) ** 2
    Nh = Nq + 3 * (N + 1)
    if not (Nq <= 16 and Nh <= 32):
        _replay_fp64_pieces(Nq, Nh)
        return
    evaluated, delivered = _replay_fp64_diagonals(Nq, Nh)
    want = {frozenset((l, m)) for l in range(Nq) for m in range(Nh) if m != l}
    assert set(evaluated) == want and all(v == 1 for v in evaluated.values())
    assert len(delivered) == len(want) and all(v == 1 for v in delivered.values())


def _replay_fp32_offsets(Nq, Nh, LPE=8):
    """The FP32 stage kernel's unique-pair schedule (esdg_stage2.cuh,
    stage2_unique_pairs, and the host tables of pack_ops2_t), for rules with
    Nq = 2 LPE: lane b owns rows b + LPE i (slots i < 2 volume rows, the
    slots above face rows); offset 0 pairs its two volume rows; at offset s
    the lane pairs its volume rows with the partner row m = (b + s) mod LPE +
    LPE j of slot j (volume slots at s = 1..LPE/2, where at s = LPE/2 lanes
    b < LPE/2 keep (i, j) in {(0,0), (1,1)} and the others {(0,1), (1,0)};
    face slots at s = 0..LPE-1, m < Nh), and row m's share of slot j comes to
    lane c from lane (c - s) mod LPE.  Returns the evaluated pairs and the
    shares delivered per (pair, receiving row)."""
    RPL = (Nh + LPE - 1) // LPE
    VS = Nq // LPE
    assert VS == 2
    evaluated, delivered = {}, {}

    def step(s, j, half):
        sent = {}
        for b in range(LPE):
            m = (b + s) % LPE + LPE * j
            pairs = []
            for i in range(VS):
                l = b + LPE * i
                take = m < Nh
                if half:
                    take = take and ((b < LPE // 2) == (i == j))
                if take and l != m:
                    key = frozenset((l, m))
                    evaluated[key] = evaluated.get(key, 0) + 1
                    pairs.append((l, m))
            sent[b] = pairs
        for c in range(LPE):
            row = c + LPE * j
            for (l, m) in sent[(c - s) % LPE]:
                assert m == row, "a partner share reached the wrong row"
                delivered[(l, m)] = delivered.get((l, m), 0) + 1

    for b in range(LPE):                          # offset 0: rows b and b + LPE of one lane
        key = frozenset((b, b + LPE))
        evaluated[key] = evaluated.get(key, 0) + 1
        delivered[(b, b + LPE)] = delivered.get((b, b + LPE), 0) + 1
    for s in range(1, LPE // 2 + 1):
        for j in range(VS):
            step(s, j, s == LPE // 2)
    for s in range(LPE):
        for j in range(VS, RPL):
            step(s, j, False)
    return evaluated, delivered


@pytest.mark.parametrize("N, rule", [(4, "symmetric"), (3, "collapsed")])
def test_fp32_kernel_unique_pairs_cover_each_pair_once(N, rule):
    """The FP32 stage kernel's offset schedule for the 16-point volume rules,
    replayed on the host: every non-zero pair of Q_skew (volume x volume,
    volume x face) is evaluated exactly once, by the lane of a volume row,
    and the partner row's share reaches that row exactly once."""
    Nq = 16
    Nh = Nq + 3 * (N + 1)
    evaluated, delivered = _replay_fp32_offsets(Nq, Nh)
    want = {frozenset((l, m)) for l in range(Nq) for m in range(Nh) if m != l}
    assert set(evaluated) == want and all(v == 1 for v in evaluated.values())
    assert len(delivered) == len(want) and all(v == 1 for v in delivered.values())


@pytest.mark.parametrize("Nq", [6, 10, 18, 22, 34])
def test_fp64_sbp_kernel_pair_pieces(Nq):
    """The FP64 DG-SBP kernel's split of the Nq x Nq pairs into 32 pieces of
    PL (esdg_sbp.cuh), replayed on the host: every pair is evaluated once, a
    piece files at most PR partial rows, and the lanes that row l's owner
    reads back, l Nq / PL .. ((l+1) Nq - 1) / PL, hold all of row l's pieces."""
    PL = (Nq * Nq + 31) // 32
    PR = (PL + Nq - 2) // Nq + 1
    seen, filed = {}, {}
    for lane in range(32):
        p0, p1 = lane * PL, min(lane * PL + PL, Nq * Nq)
        r, m, slot = (p0 // Nq, p0 % Nq, 0) if p0 < p1 else (0, 0, 0)
        for it in range(PL):
            if p0 + it < p1:
                seen[(r, m)] = seen.get((r, m), 0) + 1
                m += 1
                if m == Nq or p0 + it + 1 == p1:
                    filed.setdefault(r, []).append(lane)
                    slot += 1
                    assert slot <= PR
                    if m == Nq and r + 1 < Nq:
                        m, r = 0, r + 1
    assert seen == {(r, m): 1 for r in range(Nq) for m in range(Nq)}
    for l in range(Nq):
        k0, k1 = (l * Nq) // PL, ((l + 1) * Nq - 1) // PL
        assert set(filed[l]) <= set(range(k0, k1 + 1)) and 0 <= k0 <= k1 < 32


@pytest.mark.parametrize("nx, ny, expect", [(512, 512, "at"), (512, 513, "over")])
def test_noalloc_size_limit_is_checked_on_the_host(nx, ny, expect):
    # N = 3 with the collapsed rule has Nq = 16 volume points: 512 x 512 quads
    # give K Nq = 2^23, exactly the static scratch's capacity; one more row of
    # quads is over it.  The limit is checked before the attach check and
    # before any CUDA call, so an unattached context shows which side it is on.
    lib, rc, h = _build(N=3, nx=nx, ny=ny, rule=esdg.ESDG_RULE_COLLAPSED)
    assert rc == 0
    try:
        S, M = ctypes.c_double(), ctypes.c_double()
        r = lib.esdg_entropy_noalloc(h, None, ctypes.byref(S), ctypes.byref(M))
        if expect == "at":
            assert r == esdg.ESDG_ESTATE, lib.esdg_last_error(h)
        else:
            assert r == esdg.ESDG_EINVAL
            assert b"exceeds the static scratch limit" in lib.esdg_last_error(h)
    finally:
        lib.esdg_destroy(h)


@pytest.mark.parametrize("N,rule,precision,mass,dense,ok", [
    (4, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_TENSOR, True),
    (3, esdg.ESDG_RULE_COLLAPSED, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_TENSOR, True),
    (5, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_TENSOR, False),
    (4, esdg.ESDG_RULE_COLLAPSED, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_TENSOR, False),
    (2, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP64, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_TENSOR, False),
    (2, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_WEIGHT_ADJUSTED, esdg.ESDG_DENSE_TENSOR, False),
    (5, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_AUTO, True),
    (2, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP64, esdg.ESDG_MASS_EXACT, esdg.ESDG_DENSE_SIMT, True),
    (2, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, 3, False),
    (2, esdg.ESDG_RULE_SYMMETRIC, esdg.ESDG_FP32, esdg.ESDG_MASS_EXACT, -1, False),
])
def test_dense_operator_kind_is_validated(N, rule, precision, mass, dense, ok):
    """The tensor-core form of the dense contractions exists for the FP32
    modal path with the stored inverse where Np <= 16 and Nq <= 16; a request
    for it elsewhere, or an unknown kind, is refused with ESDG_EINVAL."""
    lib, rc, h = _build(N=N, nx=4, ny=4, warp=0.05, rule=rule, precision=precision, mass=mass, dense=dense)
    if ok:
        assert rc == 0 and h.value
        lib.esdg_destroy(h)
    else:
        assert rc == esdg.ESDG_EINVAL and not h.value


def test_tensor_core_context_keeps_the_fp32_pipe_operators():
    """A tensor-core context stores its operators in both layouts (the
    tensor-core B blocks for its own kernel, the FP32-pipe layout for
    ensembles): its footprint exceeds the FP32-pipe context's by a few tens
    of KB only."""
    sizes = []
    for dense in (esdg.ESDG_DENSE_SIMT, esdg.ESDG_DENSE_TENSOR):
        lib, rc, h = _build(N=4, nx=16, ny=16, warp=0.05, rule=esdg.ESDG_RULE_SYMMETRIC, precision=esdg.ESDG_FP32,
                            dense=dense)
        assert rc == 0
        nb = ctypes.c_size_t()
        assert lib.esdg_sizes(h, None, None, None, None, ctypes.byref(nb)) == 0
        sizes.append(nb.value)
        lib.esdg_destroy(h)
    assert 0 < sizes[1] - sizes[0] < 64 * 1024
