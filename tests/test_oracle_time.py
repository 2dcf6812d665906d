"""Pins of the oracle's time stepping and periodic solution (Sec. 2, Eqs. 1-3):
closed forms of the linear periodic implicit-Euler scheme, brute-force Newton
on the whole periodic system, and invariants of the periodic solution."""

import numpy as np
import pytest

from oracle.fem import FEModel
from oracle.periodic import bruteforce_periodic, linear_periodic_dft, linear_periodic_phasor
from oracle.stepping import one_period, propagate, steady_state_by_stepping
from synth import workload


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def tiny():
    p = workload("tiny")
    return p, FEModel(p)


@pytest.fixture(scope="module")
def tiny_linear():
    p = workload("tiny", linear_sheath=True)
    return p, FEModel(p)


def test_linear_closed_forms_agree_with_stepping(tiny_linear):
    p, m = tiny_linear
    traj, periods = steady_state_by_stepping(m, p.N, p.n_fine, p.T, tol=1e-13)
    u_dft = linear_periodic_dft(m, p.N, p.n_fine, p.T)
    u_ph = linear_periodic_phasor(m, p.N, p.n_fine, p.T)
    assert rel(u_dft, u_ph) < 1e-12
    assert rel(traj[:-1], u_dft) < 1e-10


def test_linear_closed_form_small_mesh():
    p = workload("small", linear_sheath=True)
    m = FEModel(p)
    traj, _ = steady_state_by_stepping(m, p.N, p.n_fine, p.T, tol=1e-13)
    assert rel(traj[:-1], linear_periodic_phasor(m, p.N, p.n_fine, p.T)) < 1e-10


def test_bruteforce_periodic_equals_stepping(tiny):
    p, m = tiny
    u_bf = bruteforce_periodic(m, p.N, p.n_fine, p.T)
    traj, _ = steady_state_by_stepping(m, p.N, p.n_fine, p.T, tol=1e-13)
    assert rel(traj, u_bf) < 1e-10
    # periodicity residual of the final state
    assert np.linalg.norm(traj[-1] - traj[0]) <= 1e-10 * np.linalg.norm(traj[0])


def test_half_wave_antisymmetry(tiny):
    """Odd-harmonic excitation and the odd map u -> K(u)u give u^{m+L/2} = -u^m."""
    p, m = tiny
    u = bruteforce_periodic(m, p.N, p.n_fine, p.T)[:-1]
    L = u.shape[0]
    assert rel(u[L // 2:], -u[:L // 2]) < 1e-10


def test_energy_identity_linear(tiny_linear):
    """Periodic IE: sum f.du = sum du'M du/dt + 1/2 sum du'K du (telescoping)."""
    p, m = tiny_linear
    u = linear_periodic_dft(m, p.N, p.n_fine, p.T)
    L = u.shape[0]
    dt = p.T / L
    lhs = rhs = 0.0
    for k in range(L):
        du = u[(k + 1) % L] - u[k]
        lhs += m.f((k + 1) * dt) @ du
        rhs += du @ (m.M @ du) / dt + 0.5 * du @ (m.K_lin @ du)
    assert lhs == pytest.approx(rhs, rel=1e-10)
    assert rhs > 0


def test_energy_inequality_nonlinear(tiny):
    """Convex magnetic energy: the source's work bounds the eddy-current loss."""
    p, m = tiny
    u = bruteforce_periodic(m, p.N, p.n_fine, p.T)
    dt = p.T / (u.shape[0] - 1)
    work = loss = 0.0
    for k in range(u.shape[0] - 1):
        du = u[k + 1] - u[k]
        work += m.f((k + 1) * dt) @ du
        loss += du @ (m.M @ du) / dt
    assert work >= loss > 0


def test_propagator_concatenates(tiny):
    """F over two subintervals equals one period's trajectory at T_2."""
    p, m = tiny
    u0 = np.random.default_rng(0).standard_normal(m.ndof) * 1e-7
    traj = one_period(m, u0, p.N, p.n_fine, p.T)
    u = propagate(m, 1, u0, p.N, p.n_fine, p.T)
    u = propagate(m, 2, u, p.N, p.n_fine, p.T)
    assert np.array_equal(u, traj[2 * p.n_fine])
