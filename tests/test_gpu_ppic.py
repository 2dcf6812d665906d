"""PP-IC (Eq. 5) on the GPU against the oracle, through the C ABI.

The handle keeps U_0..U_N; set_state sets U_N = U_0.  One iteration is
compared with the oracle's coarse sweep from the same states (two iterations
in a row, so the end-of-period state the first one leaves behind is checked
through the second one's start value), then the whole solve from rest, then
the PP-PC / PP-IC comparison on the paper-shaped case of Sec. 4.
"""

import os

import numpy as np
import pytest

from oracle.fem import FEModel
from oracle.pppc import ppic as oracle_ppic
from oracle.pppc import ppic_update
from oracle.pppc import rel_res as oracle_rel_res
from oracle.stepping import fine_sweep, one_period
from synth import workload

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module", autouse=True)
def library():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_13076_gb300 import _lib
    from paper_1905_13076_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def second_period_states(prob):
    m = FEModel(prob)
    traj = one_period(m, np.zeros(m.ndof), prob.N, prob.n_fine, prob.T)
    traj = one_period(m, traj[-1], prob.N, prob.n_fine, prob.T)
    U = np.zeros((prob.N, prob.mesh.n_nodes))
    U[:, m.free] = traj[:-1:prob.n_fine]
    return U


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_ppic_iterations_match_oracle_sweep(name):
    from paper_1905_13076_gb300 import from_problem

    prob = workload(name)
    m = FEModel(prob)
    free = prob.mesh.dirichlet == 0
    U0 = second_period_states(prob)
    # perturb the start so that U_N = U_0 is not already the fine result
    U0 *= 1.0 + 0.05 * np.cos(np.arange(prob.N))[:, None]
    Uext = np.vstack([U0[:, free], U0[:1, free]])
    with from_problem(prob, method="ppic", tol_coarse=1e-13, tol_lin=1e-12) as s:
        s.set_state(U0)
        for k in range(2):
            rr = s.iterate()
            F = fine_sweep(m, Uext[:prob.N], prob.N, prob.n_fine, prob.T)
            assert rr == pytest.approx(oracle_rel_res(Uext[:prob.N], F), rel=1e-8)
            Uext = ppic_update(m, Uext, F, prob.N, prob.T)
            got = s.get_state()
            assert rel(got[:, free], Uext[:prob.N]) < TOL64, k
            assert np.all(got[:, ~free] == 0.0)
        with pytest.raises(Exception):
            s.coarse_update(U0, U0)             # PP-IC needs U_N: not offered


def test_ppic_solve_matches_oracle():
    from paper_1905_13076_gb300 import from_problem

    prob = workload("tiny")
    m = FEModel(prob)
    ref = oracle_ppic(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=100)
    with from_problem(prob, method="ppic", tol_coarse=1e-13) as s:
        iters, rr = s.solve_periodic(tol=1e-11, kmax=100)
        U = s.get_state()
    assert ref.converged and rr <= 1e-11
    assert abs(iters - ref.iterations) <= 1
    assert rel(U[:, prob.mesh.dirichlet == 0], ref.U) < TOL64


def test_paper_shaped_pppc_and_ppic_reach_the_same_solution():
    """Sec. 4's comparison on the paper-shaped case (2269 unknowns, N = 20,
    100 fine steps per subinterval) from rest to 1e-6: both methods reach
    the same periodic steady state, and PP-PC needs no more iterations."""
    from paper_1905_13076_gb300 import from_problem

    prob = workload("paper")
    out = {}
    for method in ("pppc", "ppic"):
        with from_problem(prob, method=method) as s:
            iters, rr = s.solve_periodic(tol=1e-6, kmax=60)
            out[method] = (iters, rr, s.get_state())
        assert rr <= 1e-6
    assert out["pppc"][0] <= out["ppic"][0]
    assert rel(out["pppc"][2], out["ppic"][2]) < 1e-4
