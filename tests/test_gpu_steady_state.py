"""The medium workload's periodic steady state as the benchmark computes it
(mixed precision, tridiagonal-chunk preconditioner, quadratic predictor,
harmonic solves to 1e-3, inexact Newton schedule), checked against the FP64
oracle at full size.

The GPU solves from U = 0 to rel_res <= 1e-10.  The oracle then takes its own
fine sweep of all 64 subintervals from the GPU state U* (Eqs. 2-3, sparse LU,
one subinterval per process of a spawned pool) and one PP-PC coarse update
(Eq. 4 through Eqs. 9-14):
  * the oracle's jumps of U* give rel_res_oracle(U*), which must be at the
    level of the GPU's own test (U* is periodic for the oracle's fine scheme);
  * U1 = the oracle's next PP-PC iterate from U*.  Near the fixed point U_orc
    the iteration contracts by some rho < 1, so ||U* - U_orc|| <=
    ||U* - U1|| / (1 - rho); ||U1 - U*|| / ||U*|| <= 5e-8 keeps the error
    within the mixed path's 1e-7 for any rho <= 1/2 (PP-PC contracts by
    roughly 0.2 per iteration on this workload).
"""

import multiprocessing as mp
import os

import numpy as np
import pytest

from synth import workload

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-7


def _propagate(args):
    """Oracle fine propagator of one subinterval (a spawned worker)."""
    n, u = args
    from oracle.fem import FEModel
    from oracle.stepping import propagate

    prob = workload("medium")
    m = _propagate.model = getattr(_propagate, "model", None) or FEModel(prob)
    return n, propagate(m, n, u, prob.N, prob.n_fine, prob.T)


@pytest.fixture(scope="module")
def library():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_13076_gb300 import _lib
    from paper_1905_13076_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def test_medium_bench_options_reach_the_oracle_steady_state(library):
    from oracle.fem import FEModel
    from oracle.pppc import coarse_update, rel_res
    from paper_1905_13076_gb300 import from_problem

    prob = workload("medium")
    with from_problem(prob, precision="mixed", precond="tridiag", predictor=2, tol_coarse=1e-3,
                      newton_schedule=True) as s:
        s.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
        iters, rr = s.solve_periodic(tol=1e-10, kmax=60)
        U = s.get_state()
    assert rr <= 1e-10 and iters < 30

    m = FEModel(prob)
    Us = U[:, m.free]
    cores = max(1, min(os.cpu_count() or 1, prob.N))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map_async(_propagate, [(j + 1, Us[j]) for j in range(prob.N)], chunksize=1).get(timeout=900)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    F = np.stack([u for _, u in sorted(res, key=lambda t: t[0])])
    rr_orc = rel_res(Us, F)
    assert rr_orc <= 1e-9, rr_orc
    U1 = coarse_update(m, Us, F, prob.N, prob.T)
    step = np.linalg.norm(U1 - Us) / np.linalg.norm(Us)
    assert step <= 0.5 * TOL_MIXED, (step, rr_orc)
