"""Plain FP64 CPU oracle for the modal entropy-stable DG (ESDG) scheme for the
2D shallow water equations on curved triangles (Wu, Kubatko, Chan,
arXiv 2005.02516).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports, links or executes it,
and this package never imports the product package.  The two share no code:
every operator, mesh, geometric factor and flux here is rebuilt from the
paper's definitions, written for readability, not speed.

Modules
-------
refelem   reference triangle: basis, quadrature (collapsed, symmetric, SBP), Vq, Vf, Pq, D,
          Q-hat, Q_h (Sec. 2.1-2.3, 3.1)
mesh      structured periodic triangulation, curved warp, geometric factors,
          exact or weight-adjusted inverse mass matrices (Sec. 2.7, 2.8)
swe       entropy, entropy variables, EC flux (Sec. 2.4, 2.5, 2.8)
esdg      semi-discrete right-hand side in the literal form of eq. (dgform),
          LSRK45 time stepping (Sec. 4), diagnostics
sbp       the traditional DG-SBP scheme of Sec. 3 on SBP quadrature rules
          (refelem.sbp_quadrature): Q_SBP from Theorem 3.1, nodal unknowns
volume    dense-operator volume terms of the ESDG and traditional DG kernels
          (the cost comparison of Sec. 5.4)

Every function cites the passage of the paper it follows.  Readings of
passages that are silent, ambiguous or garbled are named where they are used.
"""

from .refelem import RefElem  # noqa: F401
from .mesh import Mesh  # noqa: F401
from .esdg import Oracle, LSRK45_A, LSRK45_B, LSRK45_C  # noqa: F401
