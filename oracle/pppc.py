"""Periodic Parareal with a periodic coarse problem (PP-PC) and its
multi-harmonic coarse solve (Secs. 2-3, Eqs. 4-14), plus PP-IC (Eq. 5) and
initial-value Parareal for comparison.

Notation follows the paper.  States U_0..U_{N-1} live at the coarse points
T_n = n T / N, with U_N identified with U_0 (periodicity).  One iteration k:

1. fine values   F_n^k = F_n(U_{n-1}^k),  n = 1..N                (Eq. 2)
2. convergence   d_n = F_n^k - U_{n mod N}^k,  rel_res = ||d|| / ||F||
3. coarse values G_n^k = G_n(U_{n-1}^k) with the implicit-Euler coarse step
                 C (G - U_{n-1}) + Kbar G = f(T_n)                   (Eq. 8)
4. right-hand side b_n = F_n^k - G_n^k                               (Eq. 7)
                 r_n = Q b_n + f(T_n),  C = M / dT,  Q = C + Kbar    (Eq. 10)
5. new iterate   solve the block-cyclic system                       (Eq. 9)
                   Q U_0 - C U_{N-1} = r_N,   Q U_n - C U_{n-1} = r_n
                 either directly (one sparse LU of the N-block matrix) or
                 by the multi-harmonic method: DFT along n, one shifted
                 system (Q - exp(-i 2 pi p / N) C) Uhat_p = rhat_p per
                 harmonic p in {-N/2+1, ..., N/2}, inverse DFT      (Eqs. 11-14)

Eq. 9 is written for a linear problem; for the nonlinear material the paper
defers the treatment of the coarse matrix (Sec. 2, end).  The reading used
here freezes, within iteration k, one linear coarse stiffness
    Kbar^k = (1/N) sum_n dK(U)U/dU |_{U = U_n^k}
(the time-averaged Newton Jacobian at the coarse points); alternatives are
the time-averaged secant matrix K(U_n^k) and the zero-field matrix K(0).  The
fixed point d = 0 (the periodic solution of the fine scheme) does not depend
on this choice; the iteration counts do.

The DFT uses the unnormalised forward transform with exp(-i 2 pi p n / N)
and the 1/N inverse; the normalisation of the paper's Fourier matrix cancels.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .stepping import fine_sweep

COARSE_LIN = ("avg_jacobian", "avg_chord", "zero_field")


@dataclass
class PPResult:
    U: np.ndarray
    iterations: int
    converged: bool
    history: list = field(default_factory=list)
    states: list = field(default_factory=list)


def coarse_matrices(model, U, N, T, lin="avg_jacobian"):
    """(Q, C, Kbar) of Eq. 10 for the frozen coarse stiffness Kbar."""
    if lin == "avg_jacobian":
        Kbar = sum(model.jacobian_K(U[n]) for n in range(N)) / N
    elif lin == "avg_chord":
        Kbar = sum(model.chord_K(U[n]) for n in range(N)) / N
    elif lin == "zero_field":
        Kbar = model.jacobian_K(np.zeros(model.ndof))
    else:
        raise ValueError(lin)
    C = model.M / (T / N)
    return (C + Kbar).tocsr(), C.tocsr(), Kbar.tocsr()


def coarse_step(Q_lu, C, x, f_new):
    """Eq. 8: one implicit-Euler step of the linear coarse propagator."""
    return Q_lu.solve(C @ x + f_new)


def block_cyclic_matrix(Q, C, N):
    """The N-block cyclic matrix of Eq. 9 (diagonal Q, sub-diagonal and corner -C)."""
    if N == 1:
        return (Q - C).tocsc()
    blocks = [[None] * N for _ in range(N)]
    for n in range(N):
        blocks[n][n] = Q
        blocks[n][(n - 1) % N] = -C
    return sp.bmat(blocks, format="csc")


def solve_block_cyclic(Q, C, r):
    """Direct sparse LU of Eq. 9; r[n] is the right-hand side of block row n."""
    N, ndof = r.shape
    x = spla.splu(block_cyclic_matrix(Q, C, N)).solve(r.reshape(-1))
    return x.reshape(N, ndof)


def harmonics(N):
    """The harmonic set P = {-N/2+1, ..., N/2} of Eq. 12 (N even)."""
    if N % 2:
        raise ValueError("N must be even")
    return list(range(-N // 2 + 1, N // 2 + 1))


def solve_multiharmonic(Q, C, r, return_spectrum=False):
    """Eqs. 11-14: DFT along n, one independent shifted complex system per
    harmonic, inverse DFT.  Returns the real time-domain solution."""
    N = r.shape[0]
    rhat = np.fft.fft(r, axis=0)
    Uhat = np.zeros_like(rhat)
    Qc = Q.astype(np.complex128)
    Cc = C.astype(np.complex128)
    for p in harmonics(N):
        z = np.exp(-2j * math.pi * p / N)
        Uhat[p % N] = spla.splu((Qc - z * Cc).tocsc()).solve(rhat[p % N])
    U = np.fft.ifft(Uhat, axis=0)
    scale = max(np.abs(U.real).max(), 1e-300)
    if np.abs(U.imag).max() > 1e-8 * scale:
        raise AssertionError("inverse DFT of a Hermitian spectrum is not real")
    return (U.real, Uhat) if return_spectrum else U.real


def jumps(U, F):
    """d_n = F_n(U_{n-1}) - U_{n mod N}, indexed by n mod N."""
    return np.roll(F, 1, axis=0) - U


def rel_res(U, F):
    return float(np.linalg.norm(jumps(U, F)) / np.linalg.norm(F))


def coarse_update(model, U, F, N, T, coarse="harmonic", lin="avg_jacobian", at="U"):
    """Steps 3-5 of one PP-PC iteration: U^{k+1} from U^k and F^k (F[j] = F_{j+1}).
    The frozen coarse stiffness is taken at the states U_n^k (at="U") or at
    the fine results F_n^k (at="F"); both sets are the N coarse points of the
    period, and at the fixed point they coincide."""
    Q, C, _ = coarse_matrices(model, U if at == "U" else F, N, T, lin)
    Q_lu = spla.splu(Q.tocsc())
    dT = T / N
    r = np.empty_like(U)
    for n in range(1, N + 1):
        fT = model.f(n * dT)
        b = F[n - 1] - coarse_step(Q_lu, C, U[n - 1], fT)
        r[n % N] = Q @ b + fT
    if coarse == "harmonic":
        return solve_multiharmonic(Q, C, r)
    if coarse == "cyclic":
        return solve_block_cyclic(Q, C, r)
    raise ValueError(coarse)


def pppc(model, N, n_fine, T, U0=None, tol=1e-12, kmax=50, coarse="harmonic",
         lin="avg_jacobian", keep_states=False, at="U", **kw):
    """PP-PC (Eq. 4) until rel_res(U^k) <= tol.  ``iterations`` is the number k
    of completed updates when the test first passes; ``U`` is that U^k."""
    U = np.zeros((N, model.ndof)) if U0 is None else np.array(U0, dtype=np.float64, copy=True)
    res = PPResult(U=U, iterations=0, converged=False)
    for k in range(kmax + 1):
        F = fine_sweep(model, U, N, n_fine, T, **kw)
        res.history.append(rel_res(U, F))
        if keep_states:
            res.states.append((U.copy(), F.copy()))
        if res.history[-1] <= tol:
            res.U, res.iterations, res.converged = U, k, True
            return res
        if k == kmax:
            break
        U = coarse_update(model, U, F, N, T, coarse, lin, at)
    res.U, res.iterations = U, kmax
    return res


def ppic_update(model, U, F, N, T, lin="avg_jacobian", at="U"):
    """One PP-IC coarse sweep (Eq. 5) on U = U_0..U_N (shape (N+1, ndof)),
    given the fine results F_n = F(U_{n-1}), n = 1..N (shape (N, ndof)): the
    new start value is the old end value, and each later value is the fine
    result corrected by the coarse propagator's change, swept forward."""
    dT = T / N
    Q, C, _ = coarse_matrices(model, U[:N] if at == "U" else F, N, T, lin)
    Q_lu = spla.splu(Q.tocsc())
    new = np.empty_like(U)
    new[0] = U[N]
    for n in range(1, N + 1):
        fT = model.f(n * dT)
        new[n] = (F[n - 1] + coarse_step(Q_lu, C, new[n - 1], fT)
                  - coarse_step(Q_lu, C, U[n - 1], fT))
    return new


def ppic(model, N, n_fine, T, tol=1e-12, kmax=200, lin="avg_jacobian", at="U", **kw):
    """PP-IC: initial-value Parareal sweeps over one period with the relaxed
    periodicity U_0^{k+1} = U_N^k (Eq. 5).  The state holds U_0..U_N; its
    residual uses the same periodic jumps as PP-PC on U_0..U_{N-1}."""
    U = np.zeros((N + 1, model.ndof))
    res = PPResult(U=U, iterations=0, converged=False)
    for k in range(kmax + 1):
        F = fine_sweep(model, U[:N], N, n_fine, T, **kw)
        res.history.append(rel_res(U[:N], F))
        if res.history[-1] <= tol:
            res.U, res.iterations, res.converged = U[:N], k, True
            return res
        if k == kmax:
            break
        U = ppic_update(model, U, F, N, T, lin, at)
    res.U, res.iterations = U[:N], kmax
    return res


def parareal_ivp(model, u0, N, n_fine, T, iterations, lin="avg_jacobian", **kw):
    """Classical initial-value Parareal on [0, T] with U_0 = u0 fixed.
    Returns the list of iterates U^0..U^iterations, each (N+1, ndof)."""
    dT = T / N
    U = np.zeros((N + 1, model.ndof))
    U[0] = u0
    Q, C, _ = coarse_matrices(model, np.repeat(U[:1], N, axis=0), N, T, lin)
    Q_lu = spla.splu(Q.tocsc())
    for n in range(1, N + 1):                      # U^0: one coarse sweep
        U[n] = coarse_step(Q_lu, C, U[n - 1], model.f(n * dT))
    out = [U.copy()]
    for _ in range(iterations):
        F = fine_sweep(model, U[:N], N, n_fine, T, **kw)
        Q, C, _ = coarse_matrices(model, U[:N], N, T, lin)
        Q_lu = spla.splu(Q.tocsc())
        new = np.empty_like(U)
        new[0] = u0
        for n in range(1, N + 1):
            fT = model.f(n * dT)
            new[n] = (F[n - 1] + coarse_step(Q_lu, C, new[n - 1], fT)
                      - coarse_step(Q_lu, C, U[n - 1], fT))
        U = new
        out.append(U.copy())
    return out
