"""Two linear-algebra identities the GPU path is built on, checked with dense
random matrices (no library, no oracle code).

1. Delta form of the coarse update (Eq. 4 with the implicit-Euler coarse
   propagator of Eq. 8 and a frozen Kbar): the block-cyclic system of Eq. 9
   for U^{k+1} equals U^{k+1}_n = F_n + W_n with, for every harmonic p,
   (Kbar + (1 - z_p) C) What_p = DFT_p[C d_{n-1}],  z_p = exp(-i 2 pi p / N),
   d_n = F_n - U_n (the jumps).
2. Time reversal of the backward (adjoint) cyclic problem
   Q W_n - C W_{n+1} = C e_{n+1}: in reversed lane order A'[j] = W_{-j mod N}
   it is the forward problem Q W'_j - C W'_{j-1} = C e'_{j-1}, so the forward
   harmonic solve applies unchanged.
"""

import numpy as np


def spd(rng, n, shift):
    A = rng.standard_normal((n, n))
    return A @ A.T + shift * np.eye(n)


def test_delta_form_equals_the_block_cyclic_coarse_system():
    rng = np.random.default_rng(0)
    n, N = 5, 6
    K, C = spd(rng, n, 1.0), spd(rng, n, 0.5)
    Q = K + C
    U = rng.standard_normal((N, n))                # U_0 .. U_{N-1}
    F = rng.standard_normal((N, n))                # F[j] = F_{j+1}(U_j), lands at U_{(j+1) mod N}
    # Eq. 4 with G_n(x) = Q^-1 (C x + f_n): U^{k+1}_n = F_n + G_n(U^{k+1}_{n-1}) - G_n(U_{n-1});
    # the sources f_n cancel, leaving one block-cyclic system
    # Q U_n - C U_{n-1} = Q F_n - C U^k_{n-1}   (n mod N)
    big = np.zeros((N * n, N * n))
    rhs = np.zeros(N * n)
    for m in range(1, N + 1):
        i = m % N
        big[i * n:(i + 1) * n, i * n:(i + 1) * n] = Q
        big[i * n:(i + 1) * n, ((m - 1) % N) * n:((m - 1) % N + 1) * n] -= C
        rhs[i * n:(i + 1) * n] = Q @ F[m - 1] - C @ U[m - 1]
    Unew = np.linalg.solve(big, rhs).reshape(N, n)
    # delta form: d_i = F_{i} - U_i with F_i = F[(i-1) mod N]
    Fs = np.roll(F, 1, axis=0)                    # Fs[i] = F_i
    d = Fs - U
    y = np.roll((C @ d.T).T, 1, axis=0)           # y[i] = C d_{i-1}
    yh = np.fft.fft(y, axis=0)
    W = np.empty_like(yh)
    for p in range(N):
        z = np.exp(-2j * np.pi * p / N)
        W[p] = np.linalg.solve(K + (1 - z) * C, yh[p])
    w = np.fft.ifft(W, axis=0).real
    assert np.allclose(Unew, Fs + w, rtol=1e-10, atol=1e-10)


def test_reversed_lanes_turn_the_backward_cyclic_problem_into_the_forward_one():
    rng = np.random.default_rng(1)
    n, N = 4, 8
    K, C = spd(rng, n, 1.0), spd(rng, n, 0.5)
    Q = K + C
    e = rng.standard_normal((N, n))
    # backward problem: Q W_n - C W_{n+1} = C e_{n+1}, cyclic
    big = np.zeros((N * n, N * n))
    rhs = np.zeros(N * n)
    for i in range(N):
        big[i * n:(i + 1) * n, i * n:(i + 1) * n] = Q
        j = (i + 1) % N
        big[i * n:(i + 1) * n, j * n:(j + 1) * n] -= C
        rhs[i * n:(i + 1) * n] = C @ e[j]
    W = np.linalg.solve(big, rhs).reshape(N, n)
    # reversed order: e'[j] = e_{-j}, forward harmonic solve of Q W'_j - C W'_{j-1} = C e'_{j-1}
    rev = (-np.arange(N)) % N
    er = e[rev]
    y = np.roll((C @ er.T).T, 1, axis=0)          # C e'_{j-1}
    yh = np.fft.fft(y, axis=0)
    Wh = np.empty_like(yh)
    for p in range(N):
        z = np.exp(-2j * np.pi * p / N)
        Wh[p] = np.linalg.solve(K + (1 - z) * C, yh[p])
    Wr = np.fft.ifft(Wh, axis=0).real
    assert np.allclose(Wr[rev], W, rtol=1e-10, atol=1e-10)   # W'_j = W_{-j}
    # and in natural order the symbol is the conjugate shift K + (1 - conj(z_p)) C
    yb = np.fft.fft(np.roll((C @ e.T).T, -1, axis=0), axis=0)
    Wb = np.empty_like(yb)
    for p in range(N):
        z = np.exp(-2j * np.pi * p / N)
        Wb[p] = np.linalg.solve(K + (1 - np.conj(z)) * C, yb[p])
    assert np.allclose(np.fft.ifft(Wb, axis=0).real, W, rtol=1e-10, atol=1e-10)
