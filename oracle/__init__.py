"""FP64 CPU oracle for the periodic eddy-current problem and PP-PC.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run this package.  The CUDA
library never routes through it, and it shares no code with that library: the
only common module is ``synth`` (seeded mesh and parameter data, none of the
method's arithmetic).

What it computes (paper: Kulchytska-Ruchka, De Gersem, Schoeps, "An efficient
steady-state analysis of the eddy current problem using a parallel-in-time
algorithm"):

* ``fem``      the semi-discrete system  M du/dt + K(u) u = f(t)  (Sec. 2, Eq. 1)
               on linear triangles, with a Brauer reluctivity in the sheath;
* ``stepping`` the fine propagator: implicit Euler with Newton and sparse LU
               (Eqs. 2-3), and sequential time stepping to periodicity;
* ``pppc``     the PP-PC iteration (Eq. 4) with the implicit-Euler coarse
               propagator (Eq. 8), its block-cyclic system (Eqs. 9-10) solved
               directly and by the multi-harmonic method (Eqs. 11-14); PP-IC
               (Eq. 5) and initial-value Parareal for comparison;
* ``periodic`` brute-force Newton on the full periodic fine system, and the
               closed-form periodic solution of the linear fine scheme;
* ``bessel``   the analytic skin-effect solution of the continuous linear
               problem in the coax geometry.

Every function is pinned by ``tests/test_oracle_*.py`` against something other
than itself (closed forms, brute force, invariants, exact identities).
"""
