"""Pins of the oracle's PP-PC iteration and multi-harmonic coarse solve
(Secs. 2-3, Eqs. 4-14) against exact identities and Parareal's mechanics."""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.fem import FEModel
from oracle.periodic import bruteforce_periodic, linear_periodic_phasor
from oracle.pppc import (block_cyclic_matrix, coarse_matrices, coarse_step, coarse_update,
                         parareal_ivp, ppic, ppic_update, pppc, solve_block_cyclic, solve_multiharmonic)
from oracle.stepping import fine_sweep, one_period
from synth import workload


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def knee_states(m, N, seed):
    """N smooth states with sheath flux densities of 0.5-2 T, plus small noise."""
    rng = np.random.default_rng(seed)
    xy = m.problem.mesh.xy[m.free]
    base = 4e-3 - np.hypot(xy[:, 0], xy[:, 1])
    a = rng.uniform(0.5, 2.0, size=(N, 1))
    return a * base[None] + 1e-7 * rng.standard_normal((N, m.ndof))


@pytest.fixture(scope="module")
def tiny():
    p = workload("tiny")
    return p, FEModel(p)


@pytest.fixture(scope="module")
def small():
    p = workload("small")
    return p, FEModel(p)


def test_multiharmonic_equals_block_cyclic_direct(small):
    """Eq. 13 block-diagonalises Eq. 9: both solves agree to round-off, and the
    solution satisfies every block row of Eq. 9."""
    p, m = small
    rng = np.random.default_rng(1)
    U = knee_states(m, p.N, 1)
    Q, C, _ = coarse_matrices(m, U, p.N, p.T)
    r = rng.standard_normal((p.N, m.ndof))
    x_dir = solve_block_cyclic(Q, C, r)
    x_mh = solve_multiharmonic(Q, C, r)
    assert rel(x_mh, x_dir) < 1e-12
    for n in range(p.N):
        row = Q @ x_mh[n] - C @ x_mh[(n - 1) % p.N] - r[n]
        assert np.linalg.norm(row) <= 1e-10 * np.linalg.norm(r[n])


def test_block_cyclic_matrix_structure(tiny):
    p, m = tiny
    Q, C, _ = coarse_matrices(m, np.zeros((p.N, m.ndof)), p.N, p.T)
    G = block_cyclic_matrix(Q, C, p.N).toarray()
    n = m.ndof
    assert np.array_equal(G[:n, :n], Q.toarray())
    assert np.array_equal(G[:n, -n:], -C.toarray())          # corner block couples U_0 to U_{N-1}
    assert np.array_equal(G[n:2 * n, :n], -C.toarray())
    assert not G[:n, n:2 * n].any()


def test_coarse_step_is_implicit_euler(tiny):
    """Eq. 8: C (G - U) + Kbar G = f(T_n)."""
    p, m = tiny
    U = knee_states(m, p.N, 2)
    Q, C, Kbar = coarse_matrices(m, U, p.N, p.T)
    x = U[1]
    f = m.f(0.007)
    G = coarse_step(spla.splu(Q.tocsc()), C, x, f)
    assert np.linalg.norm(C @ (G - x) + Kbar @ G - f) <= 1e-12 * np.linalg.norm(f)
    assert abs(C - m.M / (p.T / p.N)).max() == 0.0


def test_coarse_linearisation_readings(tiny):
    p, m = tiny
    # at U = 0 the averaged Jacobian is K with the zero-field reluctivity k1 + k3
    _, _, K0 = coarse_matrices(m, np.zeros((p.N, m.ndof)), p.N, p.T)
    mlin = FEModel(workload("tiny", linear_sheath=True))
    assert abs(K0 - mlin.K_lin).max() <= 1e-12 * abs(K0).max()
    # identical lanes: the average is that lane's Jacobian
    u = knee_states(m, 1, 4)[0]
    _, _, Kb = coarse_matrices(m, np.repeat(u[None], p.N, 0), p.N, p.T)
    J = m.jacobian_K(u)
    assert abs(Kb - J).max() <= 1e-12 * abs(J).max()


def test_coarse_update_cyclic_equals_harmonic(small):
    p, m = small
    rng = np.random.default_rng(3)
    U = knee_states(m, p.N, 3)
    F = U + rng.standard_normal((p.N, m.ndof)) * 1e-4
    a = coarse_update(m, U, F, p.N, p.T, coarse="cyclic")
    b = coarse_update(m, U, F, p.N, p.T, coarse="harmonic")
    assert rel(b, a) < 1e-12


def test_ivp_parareal_exact_after_k_iterations(tiny):
    """Initial-value Parareal: U_n^k equals the fine solution for n <= k."""
    p, m = tiny
    u0 = knee_states(m, 1, 5)[0]
    its = parareal_ivp(m, u0, p.N, p.n_fine, p.T, iterations=p.N)
    exact = one_period(m, u0, p.N, p.n_fine, p.T)[::p.n_fine]
    for k, U in enumerate(its):
        for n in range(1, min(k, p.N) + 1):
            assert np.linalg.norm(U[n] - exact[n]) <= 1e-11 * np.linalg.norm(exact[n])
    assert np.linalg.norm(its[1][2] - exact[2]) > 1e-6 * np.linalg.norm(exact[2])


def test_pppc_one_iteration_when_coarse_equals_fine():
    """Linear problem with one fine step per subinterval: G_n = F_n, so one
    PP-PC update lands on the periodic fine solution."""
    p = workload("tiny", linear_sheath=True, n_fine=1)
    m = FEModel(p)
    res = pppc(m, p.N, p.n_fine, p.T, tol=1e-12, kmax=3, keep_states=True)
    assert res.converged and res.iterations == 1
    exact = linear_periodic_phasor(m, p.N, p.n_fine, p.T)
    assert rel(res.U, exact) < 1e-11


def test_pppc_fixed_point_is_periodic_fine_solution(tiny):
    p, m = tiny
    u_bf = bruteforce_periodic(m, p.N, p.n_fine, p.T)
    for coarse in ("harmonic", "cyclic"):
        res = pppc(m, p.N, p.n_fine, p.T, tol=1e-12, kmax=40, coarse=coarse)
        assert res.converged
        assert rel(res.U, u_bf[:-1:p.n_fine]) < 1e-9


def test_pppc_converges_on_small_nonlinear(small):
    p, m = small
    res = pppc(m, p.N, p.n_fine, p.T, tol=1e-8, kmax=p.kmax)
    assert res.converged, res.history
    h = np.array(res.history)
    assert h[0] == pytest.approx(1.0)                    # U^0 = 0: all jumps are F
    assert (h[1:] < h[:-1]).all()


def test_ppic_converges_to_same_fixed_point(tiny):
    p, m = tiny
    a = pppc(m, p.N, p.n_fine, p.T, tol=1e-11, kmax=40)
    b = ppic(m, p.N, p.n_fine, p.T, tol=1e-11, kmax=200)
    assert a.converged and b.converged
    assert rel(b.U, a.U) < 1e-9
    assert b.iterations >= a.iterations


def test_linearisation_at_fine_results_keeps_the_fixed_point(tiny):
    """The coarse stiffness may be frozen at U^k or at the fine results F^k:
    at the fixed point the two coincide, so both iterations must reach the
    same periodic solution; for a linear material the frozen matrices are
    equal and so are the whole iterations."""
    p, m = tiny
    a = pppc(m, p.N, p.n_fine, p.T, tol=1e-11, kmax=40, at="U")
    b = pppc(m, p.N, p.n_fine, p.T, tol=1e-11, kmax=40, at="F")
    assert a.converged and b.converged
    assert rel(b.U, a.U) < 1e-9
    lin = workload("tiny", linear_sheath=True)
    ml = FEModel(lin)
    c = pppc(ml, lin.N, lin.n_fine, lin.T, tol=1e-30, kmax=3, at="U")
    d = pppc(ml, lin.N, lin.n_fine, lin.T, tol=1e-30, kmax=3, at="F")
    assert np.allclose(c.history, d.history, rtol=1e-12, atol=0)


def test_jump_of_zero_state_is_the_fine_sweep(tiny):
    p, m = tiny
    U = np.zeros((p.N, m.ndof))
    F = fine_sweep(m, U, p.N, p.n_fine, p.T)
    # from rest, subinterval n's end value is driven by the source on [T_{n-1}, T_n]
    assert np.all(np.linalg.norm(F, axis=1) > 0)
    # half-wave symmetry of the first sweep: F_{n+N/2}(0) = -F_n(0)
    assert rel(F[p.N // 2:], -F[:p.N // 2]) < 1e-10


def test_ppic_sweep_is_ivp_parareal_with_the_relaxed_start(tiny):
    """Eq. 5: a PP-IC sweep is one initial-value Parareal iteration whose
    start value is the previous end-of-period value U_N^k.  Started from an
    IVP-Parareal iterate U^0 (the coarse sweep from u0) whose end value is
    set to u0, one ppic_update must reproduce the next IVP-Parareal iterate
    U^1 (pinned above by its exactness for n <= k).  A wrong sign, index or
    start value in the sweep's correction term breaks the equality."""
    p, m = tiny
    u0 = knee_states(m, 1, 9)[0]
    its = parareal_ivp(m, u0, p.N, p.n_fine, p.T, iterations=1)
    U = its[0].copy()
    U[p.N] = u0                                          # relaxed start: U_0^{k+1} = U_N^k = u0
    F = fine_sweep(m, U[:p.N], p.N, p.n_fine, p.T)
    new = ppic_update(m, U, F, p.N, p.T)
    assert np.allclose(new[0], u0, rtol=0, atol=0)
    assert rel(new, its[1]) < 1e-13
    # the end value does move: the check is not vacuous
    assert rel(new[p.N], U[p.N]) > 1e-3


def test_ppic_with_coarse_equal_to_fine_is_sequential_stepping():
    """Linear material and one fine step per subinterval: the coarse step of
    Eq. 8 is the fine step, so every PP-IC sweep (Eq. 5) reduces to one
    period of sequential implicit Euler from the previous end value, and
    after k sweeps from rest U_N^k is the state after k periods."""
    p = workload("tiny", linear_sheath=True, n_fine=1)
    m = FEModel(p)
    U = np.zeros((p.N + 1, m.ndof))
    u = np.zeros(m.ndof)
    for k in range(3):
        F = fine_sweep(m, U[:p.N], p.N, p.n_fine, p.T, tol_newton=1e-13)
        U = ppic_update(m, U, F, p.N, p.T)
        traj = one_period(m, u, p.N, p.n_fine, p.T, tol_newton=1e-13)
        assert rel(U, traj) < 1e-10, k
        u = traj[-1]
