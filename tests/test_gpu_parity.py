"""GPU path vs the FP64 CPU oracle, through the C ABI.

Tolerances: relative L2 difference 1e-9 for the FP64 path and 1e-7 for the
mixed path (FP32 inner PCG/COCG), over the coarse-point states U_n and, for
the periodic solution, over every fine time level of the period.
"""

import os

import numpy as np
import pytest

from oracle.fem import FEModel
from oracle.pppc import coarse_update as oracle_coarse_update
from oracle.pppc import pppc as oracle_pppc
from oracle.pppc import rel_res as oracle_rel_res
from oracle.stepping import fine_sweep, one_period, propagate
from synth import workload

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL_MIXED = 1e-7


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


def gpu_solver(prob, **kw):
    from paper_1905_13076_gb300 import from_problem

    return from_problem(prob, **kw)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def knee_states(prob, seed):
    """Smooth states with sheath flux densities of 0.3-1.2 T (all nodes, zero
    on the Dirichlet ring).  Not in equilibrium outside the conductor, so they
    serve the linear-algebra (coarse) checks, not as initial values."""
    rng = np.random.default_rng(seed)
    xy = prob.mesh.xy
    base = 4e-3 - np.hypot(xy[:, 0], xy[:, 1])
    a = rng.uniform(0.2, 0.8, size=(prob.N, 1))
    U = a * base[None] + 1e-7 * rng.standard_normal((prob.N, xy.shape[0]))
    return U * (prob.mesh.dirichlet == 0)[None]


_TRAJ = {}


def physical_states(prob, periods=2):
    """Initial values the fine propagators meet in practice: the coarse-point
    states of the oracle's sequential time stepping from rest, taken in its
    second period (consistent with the algebraic equations outside the
    conductor)."""
    key = (prob.name, prob.N, prob.n_fine, prob.mesh.nr, prob.mesh.ntheta, periods, bool(prob.nu_model[2] == 0))
    if key not in _TRAJ:
        m = FEModel(prob)
        u = np.zeros(m.ndof)
        for _ in range(periods):
            traj = one_period(m, u, prob.N, prob.n_fine, prob.T)
            u = traj[-1]
        U = np.zeros((prob.N, prob.mesh.n_nodes))
        U[:, m.free] = traj[:-1:prob.n_fine]
        _TRAJ[key] = U
    return _TRAJ[key].copy()


def free(prob, U):
    return U[:, prob.mesh.dirichlet == 0]


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_fine_sweep_matches_oracle(name):
    prob = workload(name)
    m = FEModel(prob)
    U0 = physical_states(prob)
    with gpu_solver(prob) as s:
        F = s.propagate_fine(U0)
        st = s.stats()
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    assert rel(free(prob, F), ref) < TOL64
    for j in range(prob.N):                      # every lane on its own
        assert rel(free(prob, F)[j], ref[j]) < TOL64
    assert np.all(F[:, prob.mesh.dirichlet == 1] == 0.0)
    assert st["newton_iters"] >= prob.n_fine and st["pcg_iters"] > 0


def test_fine_sweep_from_rest_is_half_wave_antisymmetric():
    prob = workload("small")
    with gpu_solver(prob) as s:
        F = s.propagate_fine(np.zeros((prob.N, prob.mesh.n_nodes)))
    h = prob.N // 2
    assert rel(F[h:], -F[:h]) < 1e-10


@pytest.mark.parametrize("lin", ["avg_jacobian", "avg_chord", "zero_field"])
def test_coarse_update_matches_oracle(lin):
    prob = workload("small")
    m = FEModel(prob)
    rng = np.random.default_rng(3)
    U = knee_states(prob, 2)
    F = (U + 1e-5 * rng.standard_normal(U.shape)) * (prob.mesh.dirichlet == 0)[None]
    with gpu_solver(prob, tol_coarse=1e-13, coarse_lin=lin) as s:
        Unew, rr = s.coarse_update(U, F)
    # the oracle's F[j] is F_{j+1}(U_j): the same array
    ref = oracle_coarse_update(m, free(prob, U), free(prob, F), prob.N, prob.T, coarse="cyclic", lin=lin)
    assert rel(free(prob, Unew), ref) < TOL64
    assert rr == pytest.approx(oracle_rel_res(free(prob, U), free(prob, F)), rel=1e-12)


def test_pppc_small_matches_oracle():
    prob = workload("small")
    m = FEModel(prob)
    with gpu_solver(prob, tol_coarse=1e-12) as s:
        iters, rr = s.solve_periodic(tol=1e-11, kmax=40)
        U = s.get_state()
        st = s.stats()
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=40)
    assert ref.converged and rr <= 1e-11
    assert abs(iters - ref.iterations) <= 1
    assert rel(free(prob, U), ref.U) < TOL64
    assert st["pppc_iters"] == iters and st["cocg_iters"] > 0


def test_iterates_track_oracle():
    """The first PP-PC iterates (not only the fixed point) follow the oracle."""
    prob = workload("small")
    m = FEModel(prob)
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-30, kmax=3, keep_states=True)
    with gpu_solver(prob, tol_coarse=1e-13, tol_lin=1e-12) as s:
        for k in range(3):
            rr = s.iterate()
            assert rr == pytest.approx(ref.history[k], rel=1e-7, abs=1e-12)
            Uk1 = free(prob, s.get_state())
            Uref = ref.states[k + 1][0] if k + 1 < len(ref.states) else ref.U
            assert rel(Uk1, Uref) < 1e-8


def test_periodic_trajectory_over_the_period():
    """L2-over-the-period parity: a second GPU decomposition with one fine
    step per subinterval (N' = N n_fine) has the same fixed point and returns
    every fine time level; it must match the oracle's periodic trajectory."""
    prob = workload("small")
    m = FEModel(prob)
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-12, kmax=40)
    traj = one_period(m, ref.U[0], prob.N, prob.n_fine, prob.T)[:-1]       # u^0..u^{L-1}
    L = prob.N * prob.n_fine
    fine_prob = workload("small", N=L, n_fine=1)
    with gpu_solver(fine_prob, tol_coarse=1e-12) as s:
        iters, rr = s.solve_periodic(tol=1e-11, kmax=200)
        Ug = free(fine_prob, s.get_state())
    dt = prob.T / L
    l2 = lambda X: np.sqrt(dt * np.sum(X * X))
    assert l2(Ug - traj) / l2(traj) < TOL64
    # and the coarse-point states of the two decompositions agree
    assert rel(Ug[::prob.n_fine], ref.U) < TOL64


def test_mixed_precision_small():
    prob = workload("small")
    m = FEModel(prob)
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=40)
    with gpu_solver(prob, precision="mixed") as s:
        iters, rr = s.solve_periodic(tol=1e-10, kmax=60)
        U = s.get_state()
    assert rel(free(prob, U), ref.U) < TOL_MIXED


@pytest.mark.parametrize("over", [dict(N=2), dict(N=20, n_fine=5), dict(n_fine=1), dict(linear_sheath=True)])
def test_edge_shapes_match_oracle(over):
    """Smallest N, N not a power of two (the paper's N = 20), one fine step
    per subinterval, and a mesh without nonlinear elements."""
    prob = workload("tiny", **over)
    m = FEModel(prob)
    U0 = physical_states(prob)
    with gpu_solver(prob, tol_coarse=1e-13) as s:
        F = s.propagate_fine(U0)
        iters, rr = s.solve_periodic(tol=1e-11, kmax=80)
        U = s.get_state()
    assert rel(free(prob, F), fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)) < TOL64
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=80)
    assert rel(free(prob, U), ref.U) < TOL64


def test_medium_sampled_lanes():
    """Full-size medium mesh (19 801 DOFs, N = 64, 50 fine steps): sampled
    lanes of one batched fine sweep against the oracle's propagator."""
    prob = workload("medium")
    m = FEModel(prob)
    U0 = np.zeros((prob.N, prob.mesh.n_nodes))          # from rest: lanes differ by their time window
    with gpu_solver(prob) as s:
        F = s.propagate_fine(U0)
    Ff = free(prob, F)
    U0f = free(prob, U0)
    for j in (0, 37):
        ref = propagate(m, j + 1, U0f[j], prob.N, prob.n_fine, prob.T)
        assert rel(Ff[j], ref) < TOL64
    h = prob.N // 2
    assert np.all(np.isfinite(Ff))


def test_errors_are_reported():
    from paper_1905_13076_gb300 import PPPCError

    prob = workload("tiny")
    with gpu_solver(prob, max_lin=1) as s:
        with pytest.raises(PPPCError) as e:
            s.propagate_fine(physical_states(prob))
        assert e.value.status == 5                      # PPPC_ERR_LINEAR
    with gpu_solver(prob) as s:
        it, rr = s.solve_periodic(tol=1e-30, kmax=0, raise_on_fail=False)
        assert it == 0 and rr == pytest.approx(1.0)     # U = 0: all jumps are F
        with pytest.raises(PPPCError) as e:
            s.solve_periodic(tol=1e-30, kmax=1)
        assert e.value.status == 9                      # PPPC_ERR_NOT_CONVERGED
    bad = workload("tiny")
    bad.mesh.tri[0, 0] = bad.mesh.n_nodes + 3
    with pytest.raises(PPPCError) as e:
        gpu_solver(bad)
    assert e.value.status == 1


def test_device_pointers_and_stream():
    torch = pytest.importorskip("torch")
    prob = workload("tiny")
    U0 = physical_states(prob)
    stream = torch.cuda.Stream()
    with gpu_solver(prob, stream=stream) as s:
        F_host = s.propagate_fine(U0)
        with torch.cuda.stream(stream):
            F_dev = s.propagate_fine(torch.from_numpy(U0).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(F_dev.cpu().numpy(), F_host)


def test_handles_with_different_meshes_coexist():
    """The kernels' shared-memory limit is per function: a handle created
    later with a smaller mesh must not break an earlier, larger one."""
    big = gpu_solver(workload("small"))
    small = gpu_solver(workload("tiny"))
    big.iterate()
    small.iterate()
    big.iterate()
    big.close()
    small.close()


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_cold_start_at_high_current_backtracks(precision, tol):
    """40 A switched onto a cable at rest: the first Newton iterates of many
    steps overshoot into the steep part of the Brauer law and the residual
    grows, so the GPU lanes backtrack.  Each implicit-Euler step still has one
    solution, which the oracle's undamped Newton also reaches given enough
    iterations; the two sweeps must agree."""
    from synth import make_problem

    prob = make_problem("hot", 20, 40, 16, 10, 5e6, amp=(40.0,))
    m = FEModel(prob)
    with gpu_solver(prob, precision=precision) as s:
        F = s.propagate_fine(np.zeros((prob.N, prob.mesh.n_nodes)))
        st = s.stats()
    ref = fine_sweep(m, np.zeros((prob.N, m.ndof)), prob.N, prob.n_fine, prob.T, max_newton=200)
    assert rel(free(prob, F), ref) < tol
    assert st["backtracks"] > 0


def test_coarse_update_at_fine_results_matches_oracle():
    """Kbar frozen at the fine results F^k instead of U^k."""
    prob = workload("small")
    m = FEModel(prob)
    rng = np.random.default_rng(3)
    U = knee_states(prob, 2)
    F = knee_states(prob, 7) + 1e-6 * rng.standard_normal(U.shape) * (prob.mesh.dirichlet == 0)[None]
    with gpu_solver(prob, tol_coarse=1e-13, coarse_at="F") as s:
        Unew, _ = s.coarse_update(U, F)
    ref = oracle_coarse_update(m, free(prob, U), free(prob, F), prob.N, prob.T, coarse="cyclic", at="F")
    ref_u = oracle_coarse_update(m, free(prob, U), free(prob, F), prob.N, prob.T, coarse="cyclic", at="U")
    assert rel(free(prob, Unew), ref) < TOL64
    assert rel(ref_u, ref) > 1e-6             # the two linearisations do differ here


def test_pppc_at_fine_results_matches_oracle():
    prob = workload("tiny")
    m = FEModel(prob)
    with gpu_solver(prob, tol_coarse=1e-12, coarse_at="F") as s:
        iters, rr = s.solve_periodic(tol=1e-11, kmax=40)
        U = s.get_state()
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=40, at="F")
    assert ref.converged and rr <= 1e-11
    assert abs(iters - ref.iterations) <= 1
    assert rel(free(prob, U), ref.U) < TOL64


def test_inexact_newton_schedule_keeps_the_fixed_point():
    """newton_schedule = 1 propagates early iterates with a looser Newton
    tolerance; the periodic solution it converges to is the oracle's."""
    prob = workload("small")
    m = FEModel(prob)
    with gpu_solver(prob, tol_coarse=1e-12, newton_schedule=True) as s:
        iters, rr = s.solve_periodic(tol=1e-11, kmax=40)
        U = s.get_state()
        st = s.stats()
    with gpu_solver(prob, tol_coarse=1e-12) as s:
        s.solve_periodic(tol=1e-11, kmax=40)
        st0 = s.stats()
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=40)
    assert rr <= 1e-11
    assert rel(free(prob, U), ref.U) < TOL64
    assert st["newton_iters"] < st0["newton_iters"]


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("mixed", TOL_MIXED)])
def test_tridiagonal_chunk_preconditioner_matches_oracle(precision, tol):
    """precond = tridiag changes only the fine PCG's preconditioner: the fine
    sweep and the periodic solution are the oracle's, with fewer PCG
    iterations."""
    prob = workload("small")
    m = FEModel(prob)
    U0 = physical_states(prob)
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    with gpu_solver(prob, precision=precision, precond="tridiag", tol_lin=1e-12 if precision == "fp64" else 1e-6) as s:
        F = s.propagate_fine(U0)
        pcg_tri = s.stats()["pcg_iters"]
    with gpu_solver(prob, precision=precision, tol_lin=1e-12 if precision == "fp64" else 1e-6) as s:
        s.propagate_fine(U0)
        pcg_jac = s.stats()["pcg_iters"]
    assert rel(free(prob, F), ref) < tol
    assert pcg_tri < pcg_jac
    with gpu_solver(prob, precision=precision, precond="tridiag", tol_coarse=1e-12) as s:
        iters, rr = s.solve_periodic(tol=1e-11 if precision == "fp64" else 1e-9, kmax=40)
        U = s.get_state()
    pp = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=40)
    assert rel(free(prob, U), pp.U) < tol


def test_quadratic_predictor_matches_oracle():
    """predictor = 2 starts each step's Newton from the quadratic
    extrapolation: only the Newton path changes, not the steps' solutions."""
    prob = workload("small")
    m = FEModel(prob)
    U0 = physical_states(prob)
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    with gpu_solver(prob, predictor=2, tol_lin=1e-12) as s:
        F = s.propagate_fine(U0)
        n2 = s.stats()["newton_iters"]
    with gpu_solver(prob, predictor=1, tol_lin=1e-12) as s:
        s.propagate_fine(U0)
        n1 = s.stats()["newton_iters"]
    assert rel(free(prob, F), ref) < TOL64
    assert n2 <= n1


def test_device_wait_times_out_and_the_context_survives(library):
    """A device wait on a flag that nothing sets runs out after the library's
    2 s limit and reports PPPC_ERR_TIMEOUT; the context stays usable."""
    import time

    t0 = time.perf_counter()
    st = library.pppc_selftest_wait_timeout(None)
    dt = time.perf_counter() - t0
    assert st == 8, library.pppc_status_string(st)       # PPPC_ERR_TIMEOUT
    assert 1.5 < dt < 30.0
    prob = workload("tiny")
    with gpu_solver(prob) as s:
        iters, rr = s.solve_periodic(tol=1e-10, kmax=40)
    assert rr <= 1e-10


def test_kernels_report_sm103(library):
    """The loaded library's kernels were built for GB300 (sm_103a): the CUDA
    runtime reports binaryVersion 103 for them."""
    import ctypes

    v = ctypes.c_int32(0)
    assert library.pppc_binary_version(ctypes.byref(v)) == 0
    assert v.value == 103


def test_fine_window_matches_oracle_steps():
    """A window of the fine sweep: every subinterval j+1 marches levels
    first..first+count from the given state.  The oracle takes the same
    implicit-Euler steps (Eq. 3) at the same global time levels; chained
    windows reproduce the whole sweep."""
    from oracle.stepping import ie_step

    prob = workload("small")
    m = FEModel(prob)
    U0 = physical_states(prob)
    first, count = 7, 5
    dt = prob.T / (prob.N * prob.n_fine)
    ref = np.empty((prob.N, m.ndof))
    for j in range(prob.N):
        u = U0[j, m.free].copy()
        for q in range(count):
            s = j * prob.n_fine + first + q + 1
            u, _ = ie_step(m, u, s * dt, dt)
        ref[j] = u
    with gpu_solver(prob, tol_lin=1e-12) as s:
        Fw = s.propagate_fine_window(U0, first, count)
        assert s.stats()["fine_steps"] == count
        assert rel(free(prob, Fw), ref) < TOL64
        full = s.propagate_fine(U0)
        a = s.propagate_fine_window(U0, 0, first)
        b = s.propagate_fine_window(a, first, prob.n_fine - first)
        assert rel(free(prob, b), free(prob, full)) < TOL64
        for bad in [(-1, 2), (0, 0), (prob.n_fine - 1, 2)]:
            with pytest.raises(Exception):
                s.propagate_fine_window(U0, *bad)


@pytest.mark.parametrize("precision,tol,lanes", [("fp64", TOL64, -1), ("fp64", TOL64, 2), ("fp64", TOL64, 4),
                                                 ("fp64", TOL64, 16), ("mixed", TOL_MIXED, 4),
                                                 ("mixed", TOL_MIXED, 8), ("mixed", TOL_MIXED, 16)])
def test_lane_teams_match_oracle(precision, tol, lanes):
    """The fine sweep split into lane teams (every team of `lanes` lanes runs
    on its own share of the SMs) computes the same propagators (Eqs. 2-3) for
    every split; -1 is one team over all lanes."""
    prob = workload("small")
    m = FEModel(prob)
    U0 = physical_states(prob)
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    with gpu_solver(prob, precision=precision, lane_team=lanes, tol_lin=1e-12 if precision == "fp64" else 1e-6,
                    tol_newton=1e-10) as s:
        F = s.propagate_fine(U0)
        plan = s.fine_plan()
        st = s.stats()
    assert rel(free(prob, F), ref) < tol
    assert plan["lanes_per_team"] == lanes
    if lanes > 0:
        assert plan["teams"] == 16 // lanes
        assert plan["blocks_min"] >= 1 and plan["blocks_max"] - plan["blocks_min"] <= 1
    # lanes needed <= lane-vectors streamed; the critical path is one team's rounds
    assert 0 < st["pcg_lane_iters"] <= st["pcg_lane_rounds"]
    assert st["pcg_iters"] * (lanes if lanes > 0 else 16) <= st["pcg_lane_rounds"]
    if lanes < 0:
        assert st["pcg_lane_rounds"] == 16 * st["pcg_iters"]


def test_lane_team_tuner_times_every_candidate():
    """With lane_team = 0 the first sweep of a new size bucket times every
    candidate split on one fine level and keeps the fastest; the sweep's
    result does not depend on it."""
    prob = workload("small", N=8, n_fine=6)
    m = FEModel(prob)
    U0 = physical_states(prob)
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    with gpu_solver(prob, precision="fp64", tol_lin=1e-12) as s:
        assert s.fine_plan()["lanes_per_team"] == 0          # not chosen before the first sweep
        F = s.propagate_fine(U0)
        plan = s.fine_plan()
    assert plan["candidates"] == [2, 4, 8]
    assert all(t > 0 for t in plan["candidate_ms"])
    best = plan["candidates"][int(np.argmin(plan["candidate_ms"]))]
    assert plan["lanes_per_team"] == best
    assert rel(free(prob, F), ref) < TOL64
    with gpu_solver(prob, precision="fp64") as s2:                # same bucket: the choice is reused
        s2.propagate_fine(U0)
        p2 = s2.fine_plan()
    assert p2["lanes_per_team"] == best and all(t == 0 for t in p2["candidate_ms"])


@pytest.mark.parametrize("precision,tol,lanes", [("fp64", TOL64, -1), ("fp64", TOL64, 0), ("mixed", TOL_MIXED, -1),
                                                 ("mixed", TOL_MIXED, 4)])
def test_multigrid_preconditioner_matches_oracle(precision, tol, lanes):
    """precond = 2 (one V-cycle of smoothed-aggregation multigrid with every
    lane's Galerkin coarse matrices) changes only how each PCG solve is
    preconditioned: the propagators (Eqs. 2-3) match the oracle, with far
    fewer PCG iterations than Jacobi."""
    prob = workload("small")
    m = FEModel(prob)
    U0 = physical_states(prob)
    ref = fine_sweep(m, free(prob, U0), prob.N, prob.n_fine, prob.T)
    kw = dict(precision=precision, lane_team=lanes, tol_lin=1e-12 if precision == "fp64" else 1e-6)
    with gpu_solver(prob, precond="amg", **kw) as s:
        F = s.propagate_fine(U0)
        plan = s.fine_plan()
        its_amg = s.stats()["pcg_lane_iters"]
    with gpu_solver(prob, precond="jacobi", **kw) as s:
        s.propagate_fine(U0)
        its_jac = s.stats()["pcg_lane_iters"]
    assert rel(free(prob, F), ref) < tol
    assert len(plan["amg_rows"]) >= 2 and plan["amg_rows"][0] == m.ndof
    assert its_amg < 0.6 * its_jac, (its_amg, its_jac)


def test_multigrid_pppc_reaches_the_oracle_fixed_point():
    """PP-PC with the multigrid-preconditioned fine solves (mixed precision)
    converges to the oracle's periodic solution."""
    prob = workload("small")
    m = FEModel(prob)
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-12, kmax=60)
    assert ref.converged
    with gpu_solver(prob, precision="mixed", precond="amg", tol_newton=1e-11) as s:
        iters, rr = s.solve_periodic(tol=1e-10, kmax=60)
        U = s.get_state()
    assert rr <= 1e-10
    assert rel(free(prob, U), ref.U) < TOL_MIXED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_multigrid_harmonic_solves_match_oracle(precision):
    """With precond = 2 each harmonic system (Eq. 13) is solved by COCG
    preconditioned with a real V-cycle of Kbar + |1 - z_p| C: the coarse update
    still equals the oracle's direct solve of the block-cyclic system (Eq. 9)
    on the small mesh, and on the medium mesh (Jacobi's iteration count grows
    with the mesh, the V-cycle's does not) it needs far fewer COCG iterations
    than with Jacobi."""
    prob = workload("small")
    m = FEModel(prob)
    rng = np.random.default_rng(3)
    U = knee_states(prob, 2)
    F = (U + 1e-5 * rng.standard_normal(U.shape)) * (prob.mesh.dirichlet == 0)[None]
    ref = oracle_coarse_update(m, free(prob, U), free(prob, F), prob.N, prob.T, coarse="cyclic")
    for pc in ("amg", "jacobi"):
        with gpu_solver(prob, precision=precision, precond=pc, tol_coarse=1e-13) as s:
            Unew, rr = s.coarse_update(U, F)
        assert rel(free(prob, Unew), ref) < TOL64, pc
    # iteration counts at a working tolerance (an FP32 V-cycle, in the mixed
    # path, is not meant for 1e-13)
    med = workload("medium")
    U = knee_states(med, 2)
    F = (U + 1e-5 * rng.standard_normal(U.shape)) * (med.mesh.dirichlet == 0)[None]
    its = {}
    for pc in ("amg", "jacobi"):
        with gpu_solver(med, precision=precision, precond=pc, tol_coarse=1e-6) as s:
            s.coarse_update(U, F)
            its[pc] = s.stats()["cocg_iters"]
    assert its["amg"] < 0.5 * its["jacobi"], its


def test_workspace_comes_from_torch_caching_allocator():
    """By default the handle's device workspace comes from PyTorch's caching
    allocator (pppc_config.alloc / free_fn): torch.cuda.memory_allocated()
    grows by about the workspace at set_mesh and drops back at close, and
    results do not depend on where the memory came from."""
    import torch

    prob = workload("small")
    U0 = physical_states(prob)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    s = gpu_solver(prob)
    grown = torch.cuda.memory_allocated() - before
    lanes = prob.N * (prob.mesh.dirichlet == 0).sum()
    assert grown > 8 * lanes * 8                        # at least 8 FP64 lane vectors
    F_torch = s.propagate_fine(U0)
    s.close()
    assert torch.cuda.memory_allocated() - before < 1024
    with gpu_solver(prob, torch_memory=False) as s2:
        assert torch.cuda.memory_allocated() - before < 1024
        F_plain = s2.propagate_fine(U0)
    assert np.array_equal(F_torch, F_plain)


def test_each_iteration_is_one_captured_graph():
    """PP-PC iterations run as one captured CUDA graph each (fine sweep,
    jumps, Kbar, DFT, harmonic solves, inverse DFT + update, commit): the same
    iterates, counts and fixed point as the host-sequenced path (taken here
    because a Newton trace is on), one graph launch per iteration, and the
    returned state is the first iterate that passed."""
    prob = workload("small")
    m = FEModel(prob)
    runs = {}
    for traced in (False, True):
        with gpu_solver(prob, lane_team=-1) as s:
            if traced:
                s.set_trace(4)
            s.set_state(np.zeros((prob.N, prob.mesh.n_nodes)))
            iters, rr = s.solve_periodic(tol=1e-10, kmax=40)
            st = s.stats()
            U = s.get_state()
            runs[traced] = (iters, rr, st, U)
    (i0, r0, s0, U0), (i1, r1, s1, U1) = runs[False], runs[True]
    assert i0 == i1 and r0 == pytest.approx(r1, rel=1e-9)
    assert s0["graph_launches"] == i0 + 1 and s1["graph_launches"] == 0
    # the graph also runs the (discarded) coarse solve of the last iteration
    assert s0["pcg_iters"] == s1["pcg_iters"] and s0["cocg_iters"] >= s1["cocg_iters"]
    assert rel(U0, U1) < 1e-12
    ref = oracle_pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-12, kmax=60)
    assert rel(free(prob, U0), ref.U) < TOL64
    # rel_res of the returned state is the one reported: no update after the last test
    with gpu_solver(prob, lane_team=-1) as s:
        s.set_state(U0)
        assert s.iterate() == pytest.approx(r0, rel=1e-6)
