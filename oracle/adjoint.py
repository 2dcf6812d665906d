"""Periodic adjoint of the period-averaged eddy-current loss and its gradient
with respect to a conducting region's conductivity and Brauer constants.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module.  Plain FP64, sparse direct solves.

The periodic fine scheme of Sec. 2 (implicit Euler, L = N n_fine steps of
dt = T / L, u^0 = u^L) has the residuals
    R_m(u) = (M/dt)(u^m - u^{m-1}) + K(u^m) u^m - f(t_m),   m = 1..L.
The loss is the implicit-Euler form of (1/T) int_0^T int sigma |dA/dt|^2:
    P = (1/T) sum_m (du^m)^T M du^m / dt,   du^m = u^m - u^{m-1}
(W/m for the 2D cross-section).  Stationarity of P - sum_m lam_m^T R_m in
u^m gives the periodic adjoint, a linear recurrence backwards in time,
    (M/dt + J_m) lam_m = (M/dt) lam_{m+1} + (2/(T dt)) M (du^m - du^{m+1}),
with J_m = d(K(u)u)/du at u^m (symmetric) and lam_{L+1} = lam_1,
du^{L+1} = du^1, and then for any parameter theta
    dP/dtheta = dP/dtheta|_u - sum_m lam_m^T dR_m/dtheta|_u.
For the conductivity s of region r (M = sum over regions of s_r M_r/s_r):
    dR_m/ds = (M_r / s) du^m / dt,   dP/ds|_u = P_r / s,
and for the Brauer constants of the nonlinear elements of region r
(nu = k1 exp(k2 b) + k3, b = |B|^2, continued past b_c by its tangent):
    dR_m/dk_i = sum_e |e| dnu/dk_i(b_e) grad N_a . grad A_e.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def eddy_loss(model, traj, T):
    """P for the periodic trajectory traj = (u^0..u^L), u^L = u^0."""
    L = traj.shape[0] - 1
    dt = T / L
    du = np.diff(traj, axis=0)                                   # du^1..du^L
    return float(np.einsum("mi,mi->", du, (model.M @ du.T).T)) / (T * dt)


def adjoint_rhs(model, traj, T):
    """g_m = (2/(T dt)) M (du^m - du^{m+1}), m = 1..L (row m-1)."""
    L = traj.shape[0] - 1
    dt = T / L
    du = np.diff(traj, axis=0)
    d = du - np.roll(du, -1, axis=0)                             # du^m - du^{m+1}, cyclic
    return (2.0 / (T * dt)) * (model.M @ d.T).T


def adjoint_matrix(model, traj, T):
    """The L-block cyclic matrix of the adjoint recurrence (row block m-1:
    M/dt + J_m on the diagonal, -M/dt on block m (mod L))."""
    L = traj.shape[0] - 1
    dt = T / L
    Mdt = (model.M / dt).tocsr()
    blocks = [[None] * L for _ in range(L)]
    for m in range(1, L + 1):
        D = Mdt + model.jacobian_K(traj[m])
        if L == 1:
            blocks[0][0] = D - Mdt
        else:
            blocks[m - 1][m - 1] = D
            blocks[m - 1][m % L] = -Mdt
    return sp.bmat(blocks, format="csc")


def solve_adjoint(model, traj, T):
    """lam_1..lam_L (rows) by one sparse direct solve of the cyclic system."""
    L = traj.shape[0] - 1
    g = adjoint_rhs(model, traj, T)
    lam = spla.splu(adjoint_matrix(model, traj, T)).solve(g.reshape(-1))
    return lam.reshape(L, model.ndof)


def region_mass(model, region):
    """M_r: the conductivity matrix of the elements of one region."""
    el = np.nonzero((model.region == region) & (model.sigma > 0.0))[0]
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    return model._scatter(el, model.sigma[el, None, None] * model.area[el, None, None] * loc[None])


def dnu_dk(model, b2, elems):
    """(3, len) derivatives of nu(b) with respect to k1, k2, k3."""
    k = model.k[elems]
    bc = np.minimum(b2, model.b2max[elems])
    over = b2 - bc
    ex = np.exp(k[:, 1] * bc)
    d1 = ex * (1.0 + k[:, 1] * over)
    d2 = k[:, 0] * ex * (bc * (1.0 + k[:, 1] * over) + over)
    d3 = np.ones_like(b2)
    return np.stack([d1, d2, d3])


def dKu_dk(model, u, region):
    """(3, ndof): d(K(u) u)/dk_i over the nonlinear elements of one region."""
    el = model.nonlinear[model.region[model.nonlinear] == region]
    out = np.zeros((3, model.ndof))
    if el.size == 0:
        return out
    gA = model.grad_A(u, el)
    b2 = np.einsum("ek,ek->e", gA, gA)
    s = np.einsum("eak,ek->ea", model.grad[el], gA)              # grad N_a . grad A
    dk = dnu_dk(model, b2, el)
    for i in range(3):
        loc = (model.area[el] * dk[i])[:, None] * s
        y = np.zeros(model.n_nodes)
        np.add.at(y, model.tri[el].ravel(), loc.ravel())
        out[i] = y[model.free]
    return out


def loss_gradient(model, traj, T, region, lam=None):
    """(P, [dP/ds, dP/dk1, dP/dk2, dP/dk3]) for region `region`, given the
    periodic trajectory; lam (L, ndof) is solved for when not given."""
    L = traj.shape[0] - 1
    dt = T / L
    if lam is None:
        lam = solve_adjoint(model, traj, T)
    P = eddy_loss(model, traj, T)
    du = np.diff(traj, axis=0)
    Mr = region_mass(model, region)
    s = float(model.problem.sigma[region])
    Pr = float(np.einsum("mi,mi->", du, (Mr @ du.T).T)) / (T * dt)
    g_s = Pr / s - float(np.einsum("mi,mi->", lam, (Mr @ du.T).T)) / (s * dt)
    g_k = np.zeros(3)
    for m in range(1, L + 1):
        g_k -= dKu_dk(model, traj[m], region) @ lam[m - 1]
    return P, np.concatenate([[g_s], g_k])


def solve_adjoint_by_periods(model, traj, T, tol=1e-13, max_periods=1000):
    """The same lam_1..lam_L by sweeping the recurrence backwards over whole
    periods, lam_{L+1} taken from the previous sweep's lam_1, until it
    repeats (the adjoint counterpart of stepping to periodic steady state;
    one sparse LU per level, reused by every sweep)."""
    L = traj.shape[0] - 1
    dt = T / L
    Mdt = (model.M / dt).tocsr()
    g = adjoint_rhs(model, traj, T)
    lus = [spla.splu((Mdt + model.jacobian_K(traj[m])).tocsc()) for m in range(1, L + 1)]
    lam_next = np.zeros(model.ndof)
    lam = np.empty((L, model.ndof))
    for _ in range(max_periods):
        x = lam_next
        for m in range(L, 0, -1):
            x = lus[m - 1].solve(Mdt @ x + g[m - 1])
            lam[m - 1] = x
        if np.linalg.norm(lam[0] - lam_next) <= tol * np.linalg.norm(lam[0]):
            return lam
        lam_next = lam[0].copy()
    raise RuntimeError("adjoint sweeps did not become periodic")
