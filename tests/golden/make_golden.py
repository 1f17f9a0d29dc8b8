"""Write the stored expected values of the long FP32/FP64 parity tests.

Runs the FP64 oracle (and only the oracle) on the manufactured-solution
workload: N=3, 64x64 quads ->
K=8192 curved triangles, manufactured solution h = 2 + 0.1 sin(pi(x+y-t)),
u = v = 0.5, b = 0.1 cos(pi x) cos(pi y), g = 1, CFL 0.25, 1000 LSRK45 steps.
Stores 4000 sampled modal coefficients of the final state (seeded indices),
the per-field L2 norms of the final state, and the L2 error against the exact
solution, to tests/golden/mms_k8192_n3_1000steps.txt.  Takes about an hour.

    python tests/golden/make_golden.py
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import Oracle  # noqa: E402
from oracle.esdg import mms_sine_forcing  # noqa: E402
from paper_2005_02516_gb300 import workloads as W  # noqa: E402


def main():
    w = W.MMS
    o = Oracle(w.N, w.nx, w.ny, ax=w.warp, ay=w.warp, g=w.g, cfl=w.cfl, forcing=mms_sine_forcing)
    xb, yb = o.points("nodal")
    o.set_bathymetry(w.bathymetry(xb, yb))
    xq, yq = o.points("volq")
    u0 = o.init_state(w.initial(xq, yq))
    dt = o.dt()
    t0 = time.time()
    u, t = o.run(u0, w.steps, dt)
    el = time.time() - t0
    err = o.l2_error(u, lambda x, y: w.exact(x, y, t))
    rng = np.random.default_rng(W.BASE_SEED)
    idx = np.sort(rng.choice(u.size, size=4000, replace=False))
    flat = u.ravel()
    out = os.path.join(HERE, "mms_k8192_n3_1000steps.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, manufactured solution N=3, K=8192 curved, %d steps, dt=%.17g, t=%.17g\n"
                % (w.steps, dt, t))
        f.write("# written by tests/golden/make_golden.py (oracle only); %.0f s\n" % el)
        f.write("norms %s\n" % " ".join("%.17g" % np.linalg.norm(u[c]) for c in range(3)))
        f.write("l2err %s\n" % " ".join("%.17g" % e for e in err))
        for i in idx:
            f.write("%d %.17g\n" % (i, flat[i]))
    print("wrote", out, "in %.0f s" % el)


if __name__ == "__main__":
    main()
