"""Pins of the oracle's periodic adjoint (loss gradient) against finite
differences of the loss and, for a linear material, against the DFT
diagonalisation of the adjoint's cyclic recurrence."""

import copy
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.adjoint import adjoint_rhs, eddy_loss, loss_gradient, solve_adjoint, solve_adjoint_by_periods
from oracle.fem import FEModel
from oracle.periodic import bruteforce_periodic
from synth import REGION_SHEATH, make_problem, workload


def periodic(problem):
    m = FEModel(problem)
    return m, bruteforce_periodic(m, problem.N, problem.n_fine, problem.T, tol=1e-12, max_newton=80)


def scaled(problem, which, factor):
    p = copy.deepcopy(problem)
    if which == 0:
        p.sigma = np.array(p.sigma, dtype=np.float64)
        p.sigma[REGION_SHEATH] *= factor
    else:
        p.brauer = np.array(p.brauer, dtype=np.float64)
        p.brauer[REGION_SHEATH, which - 1] *= factor
    return p


def loss_of(problem):
    m, traj = periodic(problem)
    return eddy_loss(m, traj, problem.T)


@pytest.mark.parametrize("amp,bmax", [(10.0, 3.0), (60.0, 1.2)])
def test_gradient_matches_central_differences(amp, bmax):
    """dP/d(sigma, k1, k2, k3) against (P(t(1+h)) - P(t(1-h))) / (2 h t).
    In the second case part of the sheath is past the cap of the Brauer law
    (lowered to 1.2 T so that the tiny mesh reaches it)."""
    prob = make_problem("tiny", 5, 8, 4, 3, 5e6, amp=(amp,), bmax=bmax)
    m, traj = periodic(prob)
    if bmax < 3.0:
        gA = m.grad_A(traj[2], m.nonlinear)
        assert np.any((gA ** 2).sum(1) > m.b2max[m.nonlinear])
    P, grad = loss_gradient(m, traj, prob.T, REGION_SHEATH)
    assert P > 0
    theta = [prob.sigma[REGION_SHEATH], *prob.brauer[REGION_SHEATH]]
    h = 1e-5
    for i in range(4):
        fd = (loss_of(scaled(prob, i, 1 + h)) - loss_of(scaled(prob, i, 1 - h))) / (2 * h * theta[i])
        assert grad[i] == pytest.approx(fd, rel=1e-6), (i, grad[i], fd)


def test_linear_adjoint_matches_dft_diagonalisation():
    """For a linear sheath the cyclic adjoint recurrence diagonalises under
    the DFT along m with the shift of the opposite sign to the forward one:
        (K + (M/dt)(1 - exp(+i 2 pi q / L))) lamhat_q = ghat_q."""
    prob = workload("tiny", linear_sheath=True)
    m, traj = periodic(prob)
    L = traj.shape[0] - 1
    dt = prob.T / L
    lam = solve_adjoint(m, traj, prob.T)
    gh = np.fft.fft(adjoint_rhs(m, traj, prob.T), axis=0)
    K = m.K_lin.astype(np.complex128)
    M = (m.M / dt).astype(np.complex128)
    lh = np.empty_like(gh)
    for q in range(L):
        lh[q] = spla.splu((K + (1.0 - np.exp(2j * math.pi * q / L)) * M).tocsc()).solve(gh[q])
    ref = np.fft.ifft(lh, axis=0).real
    assert np.linalg.norm(lam - ref) <= 1e-10 * np.linalg.norm(ref)


def test_loss_is_the_discrete_eddy_power():
    """P equals (1/T) sum over steps of sum_e sigma |e| ... computed element by
    element from the consistent mass matrix, and scales linearly with sigma
    for a fixed trajectory."""
    prob = workload("tiny")
    m, traj = periodic(prob)
    L = traj.shape[0] - 1
    dt = prob.T / L
    P = eddy_loss(m, traj, prob.T)
    full = np.zeros((L + 1, m.n_nodes))
    full[:, m.free] = traj
    tot = 0.0
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    for e in np.nonzero(m.sigma > 0)[0]:
        d = full[1:, m.tri[e]] - full[:-1, m.tri[e]]                     # (L, 3)
        tot += m.sigma[e] * m.area[e] * np.einsum("ma,ab,mb->", d, loc, d)
    assert P == pytest.approx(tot / (prob.T * dt), rel=1e-12)
    m2 = FEModel(scaled(prob, 0, 2.0))
    assert eddy_loss(m2, traj, prob.T) == pytest.approx(2 * P, rel=1e-12)


def test_adjoint_by_periods_matches_direct_solve():
    prob = workload("tiny")
    m, traj = periodic(prob)
    a = solve_adjoint(m, traj, prob.T)
    b = solve_adjoint_by_periods(m, traj, prob.T)
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(a)
