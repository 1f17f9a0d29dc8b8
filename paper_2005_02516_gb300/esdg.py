"""Python binding of the C ABI in include/esdg.h (argument marshalling only).

Every step of the method runs in libesdg.so; this module converts arguments,
hands device memory (a torch allocation) and the current torch CUDA stream to
the library, and raises on non-zero status codes.  It fails loudly when the
library has not been built: there is no CPU fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libesdg.so")

ESDG_OK = 0
ESDG_EINVAL = -1
ESDG_ENOMEM = -2
ESDG_ECUDA = -3
ESDG_ENONPOSITIVE = -4
ESDG_ENONFINITE = -5
ESDG_ESTATE = -6
ESDG_ETIMEOUT = -7
ESDG_EBUSY = -8

ESDG_FP64 = 0
ESDG_FP32 = 1
ESDG_FORCING_NONE = 0
ESDG_FORCING_MMS_SINE = 1
ESDG_BOUNDARY_PERIODIC = 0
ESDG_BOUNDARY_WALLS = 1
ESDG_RULE_COLLAPSED = 0
ESDG_RULE_SYMMETRIC = 1
ESDG_MASS_EXACT = 0
ESDG_MASS_WEIGHT_ADJUSTED = 1
ESDG_METHOD_MODAL = 0
ESDG_METHOD_SBP = 1
ESDG_DENSE_AUTO = 0
ESDG_DENSE_SIMT = 1
ESDG_DENSE_TENSOR = 2
DENSE = {"auto": ESDG_DENSE_AUTO, "simt": ESDG_DENSE_SIMT, "tensor": ESDG_DENSE_TENSOR}
ESDG_POINTS_NODAL = 0
ESDG_POINTS_VOLQ = 1
ESDG_POINTS_FACEQ = 2
ESDG_VOLUME_DG = 0
ESDG_VOLUME_ESDG = 1
ESDG_INIT_DEPTH = 0
ESDG_INIT_SURFACE = 1

# every symbol include/esdg.h declares
EXPORTS = ["esdg_build_operators", "esdg_sizes", "esdg_attach_device", "esdg_get_points",
           "esdg_init_state", "esdg_set_bathymetry", "esdg_set_state", "esdg_copy_state",
           "esdg_rhs", "esdg_step", "esdg_step_async", "esdg_check", "esdg_entropy",
           "esdg_entropy_noalloc", "esdg_dt",
           "esdg_destroy", "esdg_last_error",
           "esdg_ensemble_create", "esdg_ensemble_autotune", "esdg_ensemble_step",
           "esdg_ensemble_step_async", "esdg_ensemble_destroy", "esdg_ensemble_error",
           "esdg_get_config", "esdg_prepare", "esdg_server_create", "esdg_server_submit", "esdg_server_query",
           "esdg_server_drain", "esdg_server_stats", "esdg_server_timing", "esdg_server_destroy",
           "esdg_volume_kernel", "esdg_volume_kernel_host", "esdg_step_host", "esdg_selftest_wait_timeout",
           "esdg_l2_error", "esdg_build_partition", "esdg_partition_info", "esdg_partition_maps",
           "esdg_get_neighbors", "esdg_project", "esdg_stage", "esdg_halo_pack", "esdg_halo_unpack"]


class EsdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("esdg error %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("precision", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("warp_ax", ctypes.c_double), ("warp_ay", ctypes.c_double),
                ("g", ctypes.c_double), ("cfl", ctypes.c_double),
                ("lax_friedrichs", ctypes.c_int), ("forcing", ctypes.c_int),
                ("mms_amp", ctypes.c_double), ("mms_bamp", ctypes.c_double),
                ("mms_u0", ctypes.c_double), ("mms_v0", ctypes.c_double),
                ("volume_rule", ctypes.c_int), ("boundary", ctypes.c_int), ("mass", ctypes.c_int),
                ("method", ctypes.c_int), ("dense", ctypes.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libesdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libesdg.so is missing at %s: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    PI, PD, PS = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "esdg_build_operators": ([ctypes.POINTER(Config), ctypes.POINTER(P)], I),
        "esdg_sizes": ([P, PI, PI, PI, PI, PS], I),
        "esdg_attach_device": ([P, P, S, P], I),
        "esdg_get_points": ([P, I, P, P], I),
        "esdg_init_state": ([P, P, P, I], I),
        "esdg_set_bathymetry": ([P, P], I),
        "esdg_set_state": ([P, P, I], I),
        "esdg_copy_state": ([P, P, I], I),
        "esdg_rhs": ([P, D, P, P], I),
        "esdg_step": ([P, I, D, PD], I),
        "esdg_step_async": ([P, I, D, D], I),
        "esdg_check": ([P], I),
        "esdg_entropy": ([P, D, PD, PD, PD], I),
        "esdg_entropy_noalloc": ([P, P, PD, PD], I),
        "esdg_dt": ([P, PD], I),
        "esdg_destroy": ([P], I),
        "esdg_last_error": ([P], ctypes.c_char_p),
        "esdg_ensemble_create": ([ctypes.POINTER(P), I, ctypes.POINTER(P)], I),
        "esdg_ensemble_autotune": ([P, PI, PI], I),
        "esdg_ensemble_step": ([P, I], I),
        "esdg_ensemble_step_async": ([P, I], I),
        "esdg_ensemble_destroy": ([P], I),
        "esdg_ensemble_error": ([P], ctypes.c_char_p),
        "esdg_get_config": ([P, ctypes.POINTER(Config)], I),
        "esdg_prepare": ([P, P, P, I], I),
        "esdg_server_create": ([S, I, P, ctypes.POINTER(P)], I),
        "esdg_server_submit": ([P, P, P, P, I, I, P, PI], I),
        "esdg_server_query": ([P, I, PI, PD, PD, PD], I),
        "esdg_server_drain": ([P, D], I),
        "esdg_server_stats": ([P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), PS, PI], I),
        "esdg_server_timing": ([P, P], I),
        "esdg_server_destroy": ([P], I),
        "esdg_volume_kernel": ([I, I, I, I, D, P, P, P, P, P], I),
        "esdg_volume_kernel_host": ([I, I, I, I, D, P, P, P, P], I),
        "esdg_step_host": ([P, P, I, D, PD, P], I),
        "esdg_selftest_wait_timeout": ([P], I),
        "esdg_l2_error": ([P, P, PD], I),
        "esdg_build_partition": ([ctypes.POINTER(Config), I, I, I, ctypes.POINTER(P)], I),
        "esdg_partition_info": ([P, PI, PI, PI, PI, PI, PS], I),
        "esdg_partition_maps": ([P, P, P, P], I),
        "esdg_get_neighbors": ([P, P], I),
        "esdg_project": ([P], I),
        "esdg_stage": ([P, I, D, D], I),
        "esdg_halo_pack": ([P, P, I, P], I),
        "esdg_halo_unpack": ([P, P, P, I], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def make_config(N, nx, ny, precision="fp64", x0=-1.0, x1=1.0, y0=-1.0, y1=1.0, warp=0.0, g=1.0, cfl=0.25,
                lax_friedrichs=True, forcing="none", mms=(0.1, 0.1, 0.5, 0.5), rule="collapsed", walls=False,
                mass="exact", method="modal", dense="auto"):
    if mass not in ("exact", "weight_adjusted"):
        raise ValueError("mass must be 'exact' or 'weight_adjusted'")
    if method not in ("modal", "sbp"):
        raise ValueError("method must be 'modal' or 'sbp'")
    if dense not in DENSE:
        raise ValueError("dense must be one of %s" % sorted(DENSE))
    cfg = Config()
    cfg.N, cfg.nx, cfg.ny = N, nx, ny
    cfg.precision = ESDG_FP32 if precision == "fp32" else ESDG_FP64
    cfg.x0, cfg.x1, cfg.y0, cfg.y1 = x0, x1, y0, y1
    cfg.warp_ax = cfg.warp_ay = warp
    cfg.g, cfg.cfl = g, cfl
    cfg.lax_friedrichs = 1 if lax_friedrichs else 0
    cfg.forcing = ESDG_FORCING_MMS_SINE if forcing == "mms_sine" else ESDG_FORCING_NONE
    cfg.mms_amp, cfg.mms_bamp, cfg.mms_u0, cfg.mms_v0 = mms
    cfg.volume_rule = ESDG_RULE_SYMMETRIC if rule == "symmetric" else ESDG_RULE_COLLAPSED
    cfg.boundary = ESDG_BOUNDARY_WALLS if walls else ESDG_BOUNDARY_PERIODIC
    cfg.mass = ESDG_MASS_WEIGHT_ADJUSTED if mass == "weight_adjusted" else ESDG_MASS_EXACT
    cfg.method = ESDG_METHOD_SBP if method == "sbp" else ESDG_METHOD_MODAL
    cfg.dense = DENSE[dense]
    return cfg


class Problem:
    """A context built on the host (operators, mesh, geometry) and not yet
    attached to device memory: what a request to the Server carries."""

    def __init__(self, N, nx, ny, **kw):
        self.lib = load_library()
        self.cfg = make_config(N, nx, ny, **kw)
        h = ctypes.c_void_p()
        rc = self.lib.esdg_build_operators(ctypes.byref(self.cfg), ctypes.byref(h))
        if rc != ESDG_OK:
            raise EsdgError(rc, self.lib.esdg_last_error(None).decode())
        self.h = h
        K, Np, Nq, Nfq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nbytes = ctypes.c_size_t()
        self.lib.esdg_sizes(h, ctypes.byref(K), ctypes.byref(Np), ctypes.byref(Nq), ctypes.byref(Nfq),
                            ctypes.byref(nbytes))
        self.K, self.Np, self.Nq, self.Nfq = K.value, Np.value, Nq.value, Nfq.value
        self.ndof = self.Nq if self.cfg.method == ESDG_METHOD_SBP else self.Np
        self.device_bytes = nbytes.value

    def points(self, kind):
        n = {ESDG_POINTS_NODAL: self.Np, ESDG_POINTS_VOLQ: self.Nq, ESDG_POINTS_FACEQ: self.Nfq}[kind]
        x = np.zeros((self.K, n))
        y = np.zeros((self.K, n))
        rc = self.lib.esdg_get_points(self.h, kind, _ptr(x), _ptr(y))
        if rc != ESDG_OK:
            raise EsdgError(rc, self.lib.esdg_last_error(self.h).decode())
        return x, y

    def release(self):
        """Hand the context over (the server owns it after a submit)."""
        h, self.h = self.h, None
        return h

    def close(self):
        if getattr(self, "h", None):
            self.lib.esdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (worker thread inside the library)."""

    def __init__(self, hbm_budget_bytes, max_active=256, stream=None):
        import torch
        self.lib = load_library()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self.lib.esdg_server_create(int(hbm_budget_bytes), max_active, stream.cuda_stream, ctypes.byref(h))
        if rc != ESDG_OK:
            raise EsdgError(rc, "esdg_server_create failed")
        self.h = h
        self._results = {}

    def submit(self, problem, b_nodal, q_volq, nsteps, surface=False):
        """Submit a Problem (ownership passes to the server); returns a ticket."""
        b = np.ascontiguousarray(b_nodal, dtype=np.float64)
        q = np.ascontiguousarray(q_volq, dtype=np.float64)
        out = np.zeros((3, problem.K, problem.ndof))
        t = ctypes.c_int()
        rc = self.lib.esdg_server_submit(self.h, problem.h, _ptr(b), _ptr(q),
                                         ESDG_INIT_SURFACE if surface else ESDG_INIT_DEPTH, nsteps, _ptr(out),
                                         ctypes.byref(t))
        if rc != ESDG_OK:
            raise EsdgError(rc, "esdg_server_submit refused the request")
        problem.release()
        self._results[t.value] = out
        return t.value

    def query(self, ticket):
        st = ctypes.c_int()
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        rc = self.lib.esdg_server_query(self.h, ticket, ctypes.byref(st), ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c))
        if rc != ESDG_OK:
            raise EsdgError(rc, "unknown ticket")
        return st.value, a.value, b.value, c.value

    def result(self, ticket):
        return self._results[ticket]

    def drain(self, timeout_s=600.0):
        rc = self.lib.esdg_server_drain(self.h, timeout_s)
        if rc != ESDG_OK:
            raise EsdgError(rc, "esdg_server_drain timed out")

    def stats(self):
        """(iterations, steps, device bytes in use, most requests advanced by one iteration)."""
        it, st, b, m = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t(), ctypes.c_int()
        self.lib.esdg_server_stats(self.h, ctypes.byref(it), ctypes.byref(st), ctypes.byref(b), ctypes.byref(m))
        return it.value, st.value, b.value, m.value

    def timing(self):
        """Seconds the server's worker spent admitting, rebuilding ensembles,
        enqueueing, waiting for the GPU and retiring results."""
        t = (ctypes.c_double * 5)()
        self.lib.esdg_server_timing(self.h, t)
        return dict(zip(("admit", "rebuild", "launch", "wait", "retire"), list(t)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.esdg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One ESDG problem on the current CUDA device.

    Device memory comes from a torch allocation handed to the library; work
    runs on torch's current stream at construction time.
    """

    def __init__(self, N, nx, ny, precision="fp64", x0=-1.0, x1=1.0, y0=-1.0, y1=1.0,
                 warp=0.0, g=1.0, cfl=0.25, lax_friedrichs=True, forcing="none",
                 mms=(0.1, 0.1, 0.5, 0.5), rule="collapsed", walls=False, mass="exact", method="modal",
                 torch_memory=True, stream=None, partition=None, dense="auto"):
        import torch
        self.lib = load_library()
        cfg = make_config(N, nx, ny, precision=precision, x0=x0, x1=x1, y0=y0, y1=y1, warp=warp, g=g, cfl=cfl,
                          lax_friedrichs=lax_friedrichs, forcing=forcing, mms=mms, rule=rule, walls=walls, mass=mass,
                          method=method, dense=dense)
        self.cfg = cfg
        h = ctypes.c_void_p()
        if partition is None:
            self._check(self.lib.esdg_build_operators(ctypes.byref(cfg), ctypes.byref(h)), None)
        else:
            # block `part` of a px x py element partition of the mesh (one solve on several GPUs)
            px, py, part = partition
            self._check(self.lib.esdg_build_partition(ctypes.byref(cfg), px, py, part, ctypes.byref(h)), None)
        self.h = h
        self.partition = partition
        K, Np, Nq, Nfq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nbytes = ctypes.c_size_t()
        self._check(self.lib.esdg_sizes(h, ctypes.byref(K), ctypes.byref(Np), ctypes.byref(Nq),
                                        ctypes.byref(Nfq), ctypes.byref(nbytes)))
        self.K, self.Np, self.Nq, self.Nfq = K.value, Np.value, Nq.value, Nfq.value
        # unknowns per element and field: modal coefficients, or the DG-SBP nodal values
        self.ndof = self.Nq if method == "sbp" else self.Np
        self.device_bytes = nbytes.value
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._buf = None
        if torch_memory:
            self._buf = torch.empty(self.device_bytes + 256, dtype=torch.uint8, device="cuda")
            base = self._buf.data_ptr()
            off = (-base) % 256
            self._check(self.lib.esdg_attach_device(h, base + off, self.device_bytes, stream.cuda_stream))
        else:
            self._check(self.lib.esdg_attach_device(h, None, 0, stream.cuda_stream))

    # -- plumbing --------------------------------------------------------------
    def _check(self, rc, h="self"):
        if rc != ESDG_OK:
            hh = self.h if h == "self" else h
            msg = self.lib.esdg_last_error(hh).decode()
            raise EsdgError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.esdg_destroy(self.h)
            self.h = None
            self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- API ---------------------------------------------------------------------
    def points(self, kind):
        n = {ESDG_POINTS_NODAL: self.Np, ESDG_POINTS_VOLQ: self.Nq, ESDG_POINTS_FACEQ: self.Nfq}[kind]
        x = np.zeros((self.K, n))
        y = np.zeros((self.K, n))
        self._check(self.lib.esdg_get_points(self.h, kind, _ptr(x), _ptr(y)))
        return x, y

    def init_state(self, b_nodal, q_volq, surface=False):
        b = None if b_nodal is None else np.ascontiguousarray(b_nodal, dtype=np.float64)
        q = np.ascontiguousarray(q_volq, dtype=np.float64)
        assert q.shape == (3, self.K, self.Nq)
        self._check(self.lib.esdg_init_state(self.h, _ptr(b), _ptr(q),
                                             ESDG_INIT_SURFACE if surface else ESDG_INIT_DEPTH))

    def set_bathymetry(self, b_nodal):
        b = np.ascontiguousarray(b_nodal, dtype=np.float64)
        self._check(self.lib.esdg_set_bathymetry(self.h, _ptr(b)))

    def set_state(self, u):
        """u: numpy (host) or torch CUDA tensor [3][K][ndof] float64."""
        on_dev = 0 if isinstance(u, np.ndarray) else 1
        if on_dev == 0:
            u = np.ascontiguousarray(u, dtype=np.float64)
        assert tuple(u.shape) == (3, self.K, self.ndof)
        self._check(self.lib.esdg_set_state(self.h, _ptr(u), on_dev))

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((3, self.K, self.ndof))
        on_dev = 0 if isinstance(out, np.ndarray) else 1
        self._check(self.lib.esdg_copy_state(self.h, _ptr(out), on_dev))
        return out

    def rhs(self, t=0.0, u_in=None, out=None):
        """du/dt as a torch CUDA tensor [3][K][ndof] float64."""
        import torch
        if out is None:
            out = torch.empty((3, self.K, self.ndof), dtype=torch.float64, device="cuda")
        self._check(self.lib.esdg_rhs(self.h, t, _ptr(u_in), _ptr(out)))
        return out

    def step(self, nsteps, dt=0.0, t=0.0):
        tt = ctypes.c_double(t)
        self._check(self.lib.esdg_step(self.h, nsteps, dt, ctypes.byref(tt)))
        return tt.value

    def step_host(self, u_in, nsteps=1, dt=0.0, t=0.0, out=None):
        """esdg_step_host: the state u_in (host [3][K][ndof] float64 in pinned
        memory, e.g. a numpy view of a torch pin_memory tensor) is read by the
        device directly, nsteps steps run and the result is written to out
        (pinned host memory; default: u_in itself).  Returns (out, t)."""
        out = u_in if out is None else out
        for a in (u_in, out):
            assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.shape == (3, self.K, self.ndof)
        tt = ctypes.c_double(t)
        self._check(self.lib.esdg_step_host(self.h, _ptr(u_in), nsteps, dt, ctypes.byref(tt), _ptr(out)))
        return out, tt.value

    def step_async(self, nsteps, dt=0.0, t=0.0):
        self._check(self.lib.esdg_step_async(self.h, nsteps, dt, t))

    def check(self):
        self._check(self.lib.esdg_check(self.h))

    def entropy(self, t=0.0, rate=True):
        S, M, R = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.esdg_entropy(self.h, t, ctypes.byref(S), ctypes.byref(M),
                                          ctypes.byref(R) if rate else None))
        return (S.value, M.value, R.value if rate else None)

    def l2_error(self, exact):
        """esdg_l2_error: per-field L2 error of the state against exact values
        (3, K, Nq) at the ESDG_POINTS_VOLQ points (numpy array or CUDA
        tensor; a numpy array is copied to the device first)."""
        import torch
        ex = torch.as_tensor(np.ascontiguousarray(exact, dtype=np.float64) if isinstance(exact, np.ndarray)
                             else exact, device="cuda", dtype=torch.float64).contiguous()
        assert tuple(ex.shape) == (3, self.K, self.Nq)
        err = (ctypes.c_double * 3)()
        self._check(self.lib.esdg_l2_error(self.h, _ptr(ex), err))
        return np.array(err[:])

    def dt(self):
        d = ctypes.c_double()
        self._check(self.lib.esdg_dt(self.h, ctypes.byref(d)))
        return d.value

    # -- per-stage stepping and the halo of an element partition --------------------
    def project(self):
        """esdg_project: u~ of the current state into the current u~ buffer."""
        self._check(self.lib.esdg_project(self.h))

    def stage(self, s, dt, t0):
        """esdg_stage: LSRK45 stage s (0..4) of the step that starts at t0."""
        self._check(self.lib.esdg_stage(self.h, s, dt, t0))

    def halo_pack(self, faces, out):
        """Face traces of faces = 4 e + f of local elements (int32 CUDA tensor)
        into out (CUDA tensor of at least len(faces) * trace_bytes bytes)."""
        self._check(self.lib.esdg_halo_pack(self.h, _ptr(faces), int(faces.numel()), _ptr(out)))

    def halo_unpack(self, buf, faces):
        """Face traces from buf (CUDA tensor) into the faces 4 g + f of ghost
        records (int32 CUDA tensor)."""
        self._check(self.lib.esdg_halo_unpack(self.h, _ptr(buf), _ptr(faces), int(faces.numel())))


def partition_layout(lib, h):
    """Host-side maps of a context built by esdg_build_partition (no device
    work): dict with K, K_global, nghost, px, py, part, trace_bytes,
    owned_gid [K], ghost_gid [G], ghost_part [G], nbr [K][3]."""
    K, Np, Nq, Nfq = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nb = ctypes.c_size_t()
    lib.esdg_sizes(h, ctypes.byref(K), ctypes.byref(Np), ctypes.byref(Nq), ctypes.byref(Nfq), ctypes.byref(nb))
    Kg, G, px, py, part = (ctypes.c_int() for _ in range(5))
    rb = ctypes.c_size_t()
    rc = lib.esdg_partition_info(h, ctypes.byref(Kg), ctypes.byref(G), ctypes.byref(px), ctypes.byref(py),
                                 ctypes.byref(part), ctypes.byref(rb))
    if rc != ESDG_OK:
        raise EsdgError(rc, lib.esdg_last_error(h).decode())
    owned = np.zeros(K.value, dtype=np.int32)
    gg = np.zeros(G.value, dtype=np.int32)
    gp = np.zeros(G.value, dtype=np.int32)
    lib.esdg_partition_maps(h, _ptr(owned), _ptr(gg), _ptr(gp))
    nbr = np.zeros((K.value, 3), dtype=np.int32)
    lib.esdg_get_neighbors(h, _ptr(nbr))
    return {"K": K.value, "K_global": Kg.value, "nghost": G.value, "px": px.value, "py": py.value,
            "part": part.value, "trace_bytes": rb.value, "owned_gid": owned, "ghost_gid": gg, "ghost_part": gp,
            "nbr": nbr}


class Ensemble:
    """Several independent FP32 problems (Solver objects on one stream)
    advanced together: one persistent launch per RK stage over all members,
    steps replayed from a captured CUDA graph."""

    def __init__(self, solvers):
        self.lib = load_library()
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        h = ctypes.c_void_p()
        rc = self.lib.esdg_ensemble_create(arr, len(self.solvers), ctypes.byref(h))
        if rc != ESDG_OK:
            raise EsdgError(rc, self.lib.esdg_ensemble_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != ESDG_OK:
            raise EsdgError(rc, self.lib.esdg_ensemble_error(self.h).decode())

    def autotune(self):
        w, o = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.esdg_ensemble_autotune(self.h, ctypes.byref(w), ctypes.byref(o)))
        return w.value, o.value

    def step(self, nsteps):
        self._check(self.lib.esdg_ensemble_step(self.h, nsteps))

    def step_async(self, nsteps):
        self._check(self.lib.esdg_ensemble_step_async(self.h, nsteps))

    def close(self):
        if getattr(self, "h", None):
            self.lib.esdg_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def volume_kernel(kind, Qx, Qy, u, g=1.0, out=None, stream=None):
    """Volume term of the cost comparison of Sec. 5.4 (esdg_volume_kernel):
    kind ESDG_VOLUME_DG (Q f) or ESDG_VOLUME_ESDG ((Q o F) 1).  Qx, Qy: (n, n);
    u: (3, K, n); float32 or float64, all torch CUDA tensors (launch on the
    current stream, or `stream`) or all numpy arrays (computed on the host,
    one thread).  Returns out."""
    lib = load_library()
    n, K = u.shape[2], u.shape[1]
    if isinstance(u, np.ndarray):
        dt = u.dtype
        prec = ESDG_FP32 if dt == np.float32 else ESDG_FP64
        Qx, Qy, u = (np.ascontiguousarray(a, dtype=dt) for a in (Qx, Qy, u))
        if out is None:
            out = np.empty_like(u)
        rc = lib.esdg_volume_kernel_host(kind, prec, n, K, g, _ptr(Qx), _ptr(Qy), _ptr(u), _ptr(out))
    else:
        import torch
        prec = ESDG_FP32 if u.dtype == torch.float32 else ESDG_FP64
        if out is None:
            out = torch.empty_like(u)
        st = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        rc = lib.esdg_volume_kernel(kind, prec, n, K, g, _ptr(Qx), _ptr(Qy), _ptr(u), _ptr(out), st)
    if rc != ESDG_OK:
        raise EsdgError(rc, "esdg_volume_kernel")
    return out
