"""Analytic time-harmonic solution of the continuous linear coax problem.

For I(t) = Im(I e^{i w t}) and a linear sheath of reluctivity nu_s, the axial
vector potential A(r) e^{i w t} of Eq. 1 (continuous in space) satisfies
    nu (1/r)(r A')' - i w sigma A = -J
with J = I / (pi R1^2) in the core and 0 elsewhere.  Piecewise:
    core        A = a0 - J r^2 / (4 nu0)
    insulation  A = a1 + b1 ln r
    sheath      A = a2 I0(g r) + b2 K0(g r),   g = sqrt(i w sigma / nu_s)
    air         A = a3 + b3 ln r
with A and nu A' continuous at R1, R2, R3 and A(R4) = 0: seven linear
equations for the seven coefficients.  The FE phasor solution of
(K + i w M) Ahat = I g converges to it at second order in the mesh size.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import iv, kv


def coax_phasor_coefficients(I, freq, sigma, nu_s, nu0, radii):
    R1, R2, R3, R4 = radii
    w = 2.0 * math.pi * freq
    J = I / (math.pi * R1 * R1)
    g = np.sqrt(1j * w * sigma / nu_s)
    A = np.zeros((7, 7), dtype=np.complex128)
    b = np.zeros(7, dtype=np.complex128)
    # unknowns: a0, a1, b1, a2, b2, a3, b3
    # R1: A continuous, nu0 A' continuous
    A[0, 0] = 1.0; A[0, 1] = -1.0; A[0, 2] = -math.log(R1); b[0] = J * R1 * R1 / (4.0 * nu0)
    A[1, 2] = nu0 / R1; b[1] = -J * R1 / 2.0
    # R2: insulation -> sheath
    A[2, 1] = 1.0; A[2, 2] = math.log(R2); A[2, 3] = -iv(0, g * R2); A[2, 4] = -kv(0, g * R2)
    A[3, 2] = nu0 / R2; A[3, 3] = -nu_s * g * iv(1, g * R2); A[3, 4] = nu_s * g * kv(1, g * R2)
    # R3: sheath -> air
    A[4, 3] = iv(0, g * R3); A[4, 4] = kv(0, g * R3); A[4, 5] = -1.0; A[4, 6] = -math.log(R3)
    A[5, 3] = nu_s * g * iv(1, g * R3); A[5, 4] = -nu_s * g * kv(1, g * R3); A[5, 6] = -nu0 / R3
    # R4: Dirichlet
    A[6, 5] = 1.0; A[6, 6] = math.log(R4)
    return np.linalg.solve(A, b), g, J


def coax_phasor(r, I, freq, sigma, nu_s, nu0, radii):
    """A(r) (complex phasor) at radii r."""
    c, g, J = coax_phasor_coefficients(I, freq, sigma, nu_s, nu0, radii)
    R1, R2, R3, R4 = radii
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros(r.shape, dtype=np.complex128)
    lr = np.log(np.where(r > 0, r, 1.0))
    core = r <= R1
    ins = (r > R1) & (r <= R2)
    sh = (r > R2) & (r <= R3)
    air = r > R3
    out[core] = c[0] - J * r[core] ** 2 / (4.0 * nu0)
    out[ins] = c[1] + c[2] * lr[ins]
    out[sh] = c[3] * iv(0, g * r[sh]) + c[4] * kv(0, g * r[sh])
    out[air] = c[5] + c[6] * lr[air]
    return out
