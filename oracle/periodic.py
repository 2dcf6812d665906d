"""Two further routes to the periodic solution of the fine scheme, used to pin
PP-PC's fixed point (Sec. 2, Eq. 1 with u(0) = u(T)).

* ``bruteforce_periodic``: Newton on all L = N n_fine implicit-Euler steps of
  one period at once, with the wrap-around u^0 = u^L, and a sparse direct
  solve of the L-block cyclic Jacobian.  Affordable at tiny sizes only.
* ``linear_periodic_dft``: for a linear material the periodic implicit-Euler
  solution diagonalises under the L-point DFT along time:
      (K + (M/dt)(1 - exp(-i 2 pi q / L))) uhat_q = fhat_q,  q = 0..L-1.
* ``linear_periodic_phasor``: for one sinusoid  I(t) = a sin(w t + phi)  with
  w T / (2 pi) integer, u^m = Im(uhat exp(i w t_m)) with
      (K + (M/dt)(1 - exp(-i w dt))) uhat = a exp(i phi) g.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def bruteforce_periodic(model, N, n_fine, T, tol=1e-11, max_newton=50, X0=None):
    """Returns (u^0..u^L) of the periodic fine solution, u^L = u^0."""
    L = N * n_fine
    dt = T / L
    ndof = model.ndof
    Mdt = (model.M / dt).tocsr()
    X = np.zeros((L, ndof)) if X0 is None else np.array(X0, dtype=np.float64)  # X[m] = u^{m+1}
    fs = np.stack([model.f((m + 1) * dt) for m in range(L)])
    scale = model.newton_scale() * math.sqrt(L)
    for _ in range(max_newton + 1):
        prev = np.roll(X, 1, axis=0)                                  # u^m (u^0 = u^L)
        R = np.stack([Mdt @ (X[m] - prev[m]) + model.Ku(X[m]) - fs[m] for m in range(L)])
        if np.linalg.norm(R) <= tol * scale:
            return np.concatenate([X[-1:], X], axis=0)
        blocks = [[None] * L for _ in range(L)]
        for m in range(L):
            blocks[m][m] = Mdt + model.jacobian_K(X[m])
            if L > 1:
                blocks[m][(m - 1) % L] = -Mdt
            else:
                blocks[m][m] = blocks[m][m] - Mdt
        J = sp.bmat(blocks, format="csc")
        X = X + spla.splu(J).solve(-R.reshape(-1)).reshape(L, ndof)
    raise RuntimeError("brute-force periodic Newton did not converge")


def linear_periodic_dft(model, N, n_fine, T):
    """Periodic implicit-Euler solution u^0..u^{L-1} for a linear model."""
    if model.nonlinear.size:
        raise ValueError("linear model required")
    L = N * n_fine
    dt = T / L
    f = np.stack([model.f(m * dt) for m in range(L)])                 # level m uses f(t_m)
    fh = np.fft.fft(f, axis=0)
    K = model.K_lin.astype(np.complex128)
    M = (model.M / dt).astype(np.complex128)
    uh = np.empty_like(fh)
    for q in range(L):
        uh[q] = spla.splu((K + (1.0 - np.exp(-2j * math.pi * q / L)) * M).tocsc()).solve(fh[q])
    return np.fft.ifft(uh, axis=0).real


def linear_periodic_phasor(model, N, n_fine, T):
    """Same solution for a single-sinusoid source, from one complex solve."""
    if model.nonlinear.size or model.amp.size != 1:
        raise ValueError("linear model with one sinusoid required")
    L = N * n_fine
    dt = T / L
    w = 2.0 * math.pi * float(model.freq[0])
    A = (model.K_lin + (1.0 - np.exp(-1j * w * dt)) * (model.M / dt)).astype(np.complex128)
    uhat = spla.splu(A.tocsc()).solve(model.amp[0] * np.exp(1j * model.phase[0]) * model.g.astype(np.complex128))
    t = np.arange(L) * dt
    return np.imag(uhat[None, :] * np.exp(1j * w * t)[:, None])
