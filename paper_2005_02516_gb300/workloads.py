"""Seeded synthetic workloads: problem definitions and random inputs.

This module holds no arithmetic of the ESDG method.  It defines three
problem configurations (mesh size, degree, warp, analytic bathymetry and
initial data as plain functions of (x, y)) and seeded random inputs.  The
tests, the benchmark and the oracle-side CPU baseline all draw their inputs
from here; the library and the oracle are each handed the same arrays or
evaluate the same analytic functions at their own points.

Base seed 20050251; instance i of an ensemble uses seed 20050251 + i.
"""

import dataclasses
import math

import numpy as np

BASE_SEED = 20050251
SYMMETRIC_POINTS = {1: 3, 2: 6, 3: 12, 4: 16, 5: 25}


def volume_points(N, rule):
    """Volume quadrature points per element for a degree and rule."""
    return SYMMETRIC_POINTS[N] if rule == "symmetric" else (N + 1) ** 2


@dataclasses.dataclass
class Workload:
    name: str
    N: int
    nx: int
    ny: int
    warp: float            # ax = ay (0 -> affine)
    g: float
    cfl: float
    steps: int
    forcing: str           # "none" or "mms_sine"
    x0: float = -1.0
    x1: float = 1.0
    y0: float = -1.0
    y1: float = 1.0
    surface_init: bool = False   # initial q[0] is the free surface H = h + b
    rule: str = "collapsed"      # volume rule: "collapsed" (exact to 2N+1) or "symmetric" (exact to 2N)

    @property
    def K(self):
        return 2 * self.nx * self.ny

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2

    @property
    def Nq(self):
        return volume_points(self.N, self.rule)

    def bathymetry(self, x, y):
        return _BATHY[self.name](x, y)

    def initial(self, x, y):
        """Initial (h or H, hu, hv) at points (x, y); shape (3, ...)."""
        return _INIT[self.name](x, y)

    def exact(self, x, y, t):
        """Closed-form solution where the workload has one (else None)."""
        f = _EXACT.get(self.name)
        return None if f is None else f(x, y, t)


def _lake_bump_bathy(x, y):
    return 0.2 * np.sin(np.pi * x) * np.sin(np.pi * y)


def _lake_bump_init(x, y):
    # H = 2 plus a Gaussian bump in h (given as the free surface)
    r2 = x * x + y * y
    return np.stack([2.0 + 0.01 * np.exp(-25.0 * r2), 0 * x, 0 * x])


def _mms_bathy(x, y):
    return 0.1 * np.cos(np.pi * x) * np.cos(np.pi * y)


def _mms_exact(x, y, t):
    h = 2.0 + 0.1 * np.sin(np.pi * (x + y - t))
    return np.stack([h, 0.5 * h, 0.5 * h])


def _dam_bathy(x, y):
    return 0.05 * np.exp(-10.0 * ((x - 0.4) ** 2 + y * y))


def _dam_init(x, y):
    r = np.sqrt(x * x + y * y)
    return np.stack([1.0 + 0.5 * np.tanh(40.0 * (0.3 - r)), 0 * x, 0 * x])


_BATHY = {"lake_bump_k128_n2": _lake_bump_bathy,
          "mms_k8192_n3": _mms_bathy,
          "dam_k131072_n4": _dam_bathy}
_INIT = {"lake_bump_k128_n2": _lake_bump_init,
         "mms_k8192_n3": lambda x, y: _mms_exact(x, y, 0.0),
         "dam_k131072_n4": _dam_init}
_EXACT = {"mms_k8192_n3": _mms_exact}

# Lake at rest plus a bump: plain FP64, N=2, 8x8 quads -> K=128 affine, g=1, H=2
# plus a bump; 200 steps at CFL 0.25.
LAKE_BUMP = Workload("lake_bump_k128_n2", N=2, nx=8, ny=8, warp=0.0, g=1.0, cfl=0.25,
                     steps=200, forcing="none", surface_init=True)
# Manufactured solution: N=3, 64x64 -> K=8192 curved, 1000 steps.
MMS = Workload("mms_k8192_n3", N=3, nx=64, ny=64, warp=0.05, g=1.0, cfl=0.25,
               steps=1000, forcing="mms_sine")
# Smoothed dam break: N=4, 256x256 -> K=131072 curved, with the 16-point
# symmetric volume rule exact to degree 2N = 8.
DAM = Workload("dam_k131072_n4", N=4, nx=256, ny=256, warp=0.05, g=1.0, cfl=0.25,
               steps=50, forcing="none", rule="symmetric")

WORKLOADS = {w.name: w for w in (LAKE_BUMP, MMS, DAM)}


def scaled(w, nx, ny=None, N=None, steps=None):
    """Same problem on another grid or degree (for small parity cases)."""
    ny = nx if ny is None else ny
    return dataclasses.replace(w, nx=nx, ny=ny, N=w.N if N is None else N,
                               steps=w.steps if steps is None else steps)


def random_modal_state(K, Np, seed, c0=2.8, amp_h=0.05, amp_m=0.05):
    """Random modal coefficients [3][K][Np]: i.i.d. normal, scaled by
    amp / (1 + mode index), with c0 added to the first (constant) mode of h.
    For an orthonormal basis on the reference triangle (area 2) the constant
    mode is 1/sqrt(2), so c0 = 2.8 gives a mean depth near 1.98 and keeps the
    depth positive everywhere for the default amplitudes."""
    rng = np.random.default_rng(seed)
    decay = 1.0 / (1.0 + np.arange(Np))
    u = rng.standard_normal((3, K, Np)) * decay[None, None, :]
    u[0] *= amp_h
    u[1:] *= amp_m
    u[0, :, 0] += c0
    return u


@dataclasses.dataclass
class Instance:
    """One member of a batched ensemble: lake at rest H = 2 plus a Gaussian bump
    on curved periodic [-1,1]^2, bathymetry amp * sin(pi x) sin(pi y)."""
    N: int
    nx: int
    amp: float
    cx: float
    cy: float
    steps: int
    warp: float = 0.05
    g: float = 1.0
    cfl: float = 0.25
    rule: str = "symmetric"

    @property
    def K(self):
        return 2 * self.nx * self.nx

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2

    def bathymetry(self, x, y):
        return self.amp * np.sin(np.pi * x) * np.sin(np.pi * y)

    def initial(self, x, y):
        r2 = (x - self.cx) ** 2 + (y - self.cy) ** 2
        return np.stack([2.0 + 0.01 * np.exp(-25.0 * r2), 0 * x, 0 * x])


def ensemble(n=64, steps=500, seed=BASE_SEED):
    """Batched ensemble: instance i draws, from seed + i, N ~ U{2,3,4},
    K ~ U{512, 2048, 8192, 32768} (nx ~ U{16, 32, 64, 128}), bathymetry
    amplitude ~ U[0.02, 0.2] and bump centre ~ U[-0.5, 0.5]^2."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed + i)
        N = int(rng.integers(2, 5))
        nx = int(rng.choice([16, 32, 64, 128]))
        amp = float(rng.uniform(0.02, 0.2))
        c = rng.uniform(-0.5, 0.5, size=2)
        out.append(Instance(N=N, nx=nx, amp=amp, cx=float(c[0]), cy=float(c[1]), steps=steps))
    return out


@dataclasses.dataclass
class Request:
    """One served solve request: arrival time, degree, grid, steps, and a
    smooth random bathymetry sum_j A_j exp(-alpha |x - c_j|^2) (4 Gaussians)
    under a lake at rest H = 2 plus a bump 0.01 exp(-25 |x - c|^2)."""
    t_arrival: float
    N: int
    nx: int
    steps: int
    amps: tuple
    centres: tuple
    bump: tuple
    alpha: float = 10.0
    warp: float = 0.05
    g: float = 1.0
    cfl: float = 0.25
    rule: str = "symmetric"

    @property
    def K(self):
        return 2 * self.nx * self.nx

    @property
    def Np(self):
        return (self.N + 1) * (self.N + 2) // 2

    def bathymetry(self, x, y):
        b = 0 * x
        for a, (cx, cy) in zip(self.amps, self.centres):
            b = b + a * np.exp(-self.alpha * ((x - cx) ** 2 + (y - cy) ** 2))
        return b

    def initial(self, x, y):
        r2 = (x - self.bump[0]) ** 2 + (y - self.bump[1]) ** 2
        return np.stack([2.0 + 0.01 * np.exp(-25.0 * r2), 0 * x, 0 * x])


def served_trace(n, rate, seed=BASE_SEED, k_range=(512, 131072), steps_range=(100, 2000), degrees=(2, 3, 4, 5)):
    """Poisson arrivals at `rate` per second; N ~ U(degrees); K log-uniform in
    k_range, rounded to the nearest 2 n^2; steps ~ U(steps_range); amplitudes
    ~ U[0, 0.2], Gaussian centres ~ U[-0.8, 0.8]^2, bump centre ~ U[-0.5, 0.5]^2."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        N = int(rng.choice(degrees))
        K = math.exp(rng.uniform(math.log(k_range[0]), math.log(k_range[1])))
        nx = max(3, int(round(math.sqrt(K / 2.0))))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        amps = tuple(float(a) for a in rng.uniform(0.0, 0.2, size=4))
        centres = tuple((float(c[0]), float(c[1])) for c in rng.uniform(-0.8, 0.8, size=(4, 2)))
        bump = tuple(float(c) for c in rng.uniform(-0.5, 0.5, size=2))
        out.append(Request(t_arrival=t, N=N, nx=nx, steps=steps, amps=amps, centres=centres, bump=bump))
    return out


def volume_ratio_inputs(n, K, seed=BASE_SEED, dtype=np.float64):
    """Inputs of the volume-kernel cost comparison (Sec. 5.4): two n x n
    operators with i.i.d. uniform [-1, 1] entries (the comparison uses random
    matrices) and a smooth-looking random state (3, K, n) with depth
    1 + U[0, 0.2] and momenta 0.1 N(0, 1)."""
    rng = np.random.default_rng(seed)
    Qx = rng.uniform(-1.0, 1.0, size=(n, n))
    Qy = rng.uniform(-1.0, 1.0, size=(n, n))
    u = np.empty((3, K, n))
    u[0] = 1.0 + 0.2 * rng.random((K, n))
    u[1:] = 0.1 * rng.standard_normal((2, K, n))
    return Qx.astype(dtype), Qy.astype(dtype), u.astype(dtype)


def lake_at_rest_table_bathymetry(x, y):
    """Bathymetry of the lake-at-rest experiment of Sec. 4.1 as printed:
    b = 0.1 sin(2 pi x) cos(2 pi x) + 0.5 (periodic on [-1,1]^2)."""
    return 0.1 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * x) + 0.5
