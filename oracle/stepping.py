"""Fine propagator and sequential time stepping (Sec. 2, Eqs. 2-3).

The fine propagator F_n solves the initial-value problem (3) on the
subinterval [T_{n-1}, T_n] with n_fine implicit-Euler steps of size
dt = T / (N n_fine) (the paper fixes only the fine step size; implicit Euler,
with the source taken at the new time level as in the coarse scheme Eq. 8, is
the reading used here).  Each step solves the nonlinear system

    R(u) = (M/dt)(u - u_prev) + K(u) u - f(t_new) = 0

by Newton's method started from u_prev, with a sparse direct solve of the
Jacobian  J = M/dt + dK(u)u/du  per iteration, until
||R||_2 <= tol_newton * ||g||_2 * sum_j |amp_j|, or until ||R|| stalls at its
rounding floor within 100 times that bound.

Time levels: the global step index s = (n-1) n_fine + m + 1 of the m-th step
of subinterval n (m = 0..n_fine-1) has t_s = s * dt.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


# Newton also stops when ||R|| no longer halves while within FLOOR_MULT of
# the tolerance: with exact linear solves that means the residual has met the
# rounding floor of its own evaluation.
STAGNATION = 0.5
FLOOR_MULT = 100.0


class NewtonError(RuntimeError):
    pass


def ie_step(model, u_prev, t_new, dt, tol_newton=1e-10, max_newton=30):
    """One implicit-Euler step with Newton; returns (u_new, newton_iterations)."""
    Mdt = model.M / dt
    fs = model.f(t_new)
    tol = tol_newton * model.newton_scale()
    u = u_prev.copy()
    r_prev = np.inf
    for it in range(max_newton + 1):
        R = Mdt @ (u - u_prev) + model.Ku(u) - fs
        r = np.linalg.norm(R)
        if r <= tol or (it > 0 and r <= FLOOR_MULT * tol and r >= STAGNATION * r_prev):
            return u, it
        r_prev = r
        if it == max_newton:
            break
        J = (Mdt + model.jacobian_K(u)).tocsc()
        u = u + spla.splu(J).solve(-R)
    raise NewtonError(f"Newton did not reach {tol:.3e} in {max_newton} iterations (t={t_new})")


def propagate(model, n, U, N, n_fine, T, tol_newton=1e-10, max_newton=30, trajectory=False):
    """F_n(U): march from T_{n-1} to T_n (n = 1..N).

    Returns the end state, or with ``trajectory=True`` the list of the
    n_fine + 1 states u(T_{n-1}), ..., u(T_n).
    """
    L = N * n_fine
    dt = T / L
    u = np.array(U, dtype=np.float64, copy=True)
    traj = [u.copy()] if trajectory else None
    for m in range(n_fine):
        s = (n - 1) * n_fine + m + 1
        u, _ = ie_step(model, u, s * dt, dt, tol_newton, max_newton)
        if trajectory:
            traj.append(u.copy())
    return traj if trajectory else u


def fine_sweep(model, U, N, n_fine, T, **kw):
    """All fine propagators of one Parareal iteration:
    out[j] = F_{j+1}(U[j]) for j = 0..N-1 (subinterval j+1 starts from U_j)."""
    return np.stack([propagate(model, j + 1, U[j], N, n_fine, T, **kw) for j in range(N)])


def one_period(model, u0, N, n_fine, T, **kw):
    """March one full period from t=0; returns the L+1 states u^0..u^L."""
    traj = [np.array(u0, dtype=np.float64, copy=True)]
    for n in range(1, N + 1):
        traj.extend(propagate(model, n, traj[-1], N, n_fine, T, trajectory=True, **kw)[1:])
    return np.stack(traj)


def steady_state_by_stepping(model, N, n_fine, T, tol=1e-10, max_periods=500, u0=None, **kw):
    """Classical approach: repeat whole periods until
    ||u(T) - u(0)|| <= tol * ||u(T)||.  Returns (trajectory over the last
    period, number of periods marched)."""
    u = np.zeros(model.ndof) if u0 is None else np.asarray(u0, dtype=np.float64)
    for k in range(1, max_periods + 1):
        traj = one_period(model, u, N, n_fine, T, **kw)
        if np.linalg.norm(traj[-1] - traj[0]) <= tol * np.linalg.norm(traj[-1]):
            return traj, k
        u = traj[-1]
    raise RuntimeError(f"no periodic steady state within {max_periods} periods")
