"""Plain, slow, FP64 CPU oracle for the ensemble lattice-Boltzmann UQ hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import, call, link or run anything in this folder.
The product package never imports it and shares no code with it: the oracle has its
own Gauss-Legendre rule, Philox generator, Legendre chaos, projection and statistics
(``uq.py``) and its own D2Q9 BGK solver in plain C (``lbm_oracle.c`` via ``lbm.py``).

Every function cites the passage of arXiv 2508.13867 it follows.  Parity status:
  * ``uq.py``: pinned by closed forms (5-point Gauss-Legendre nodes and weights,
    exactness up to degree 2n-1), published Philox4x32-10 known-answer vectors,
    discrete orthonormality, polynomial reproduction, closed-form E[K], numpy
    moments and the N^-1/2 Monte Carlo rate.
  * ``lbm_oracle.c``, Taylor-Green vortex: pinned by mass and momentum conservation,
    the rest state, the closed-form viscous decay and second-order convergence.
  * ``lbm_oracle.c``, channel walls and velocity inlet: pinned by the plane Poiseuille
    profile (mass flux of the inlet, parabolic shape, second-order convergence).
  * ``lbm_oracle.c``, obstacle forces: only a loose anchor (drag near the paper's
    deterministic value at 20 nodes per diameter); parity unpinned beyond that.
"""
from . import lbm, uq  # noqa: F401
