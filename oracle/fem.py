"""Space discretisation of the 2D A-formulation eddy-current problem (Sec. 2, Eq. 1).

    M du/dt + K(u) u = f(t),   u(0) = u(T)

u holds the nodal values of the axial magnetic vector potential A_z on linear
triangles (the paper uses the finite element method without naming the
element; linear triangles are the reading taken here).  With N_a the hat
functions of a triangle e of area |e|:

* stiffness ("curl-curl") for a linear material:
      K_ab = sum_e nu_e |e| grad N_a . grad N_b
* nonlinear material, nu = nu(|B|^2) with |B|^2 = |grad A|^2 on each element
  (Brauer law nu = k1 exp(k2 b) + k3; when a cap bmax > 0 is given, it is
  continued past b_c = bmax^2 by its tangent in b,
  nu = k1 exp(k2 b_c) (1 + k2 (b - b_c)) + k3, so nu and nu' stay continuous):
      (K(u) u)_a = sum_e |e| nu(b_e) grad N_a . grad A_e
  and its Jacobian
      J_ab = sum_e |e| [ nu grad N_a . grad N_b
                         + 2 nu'(b) (grad N_a . grad A)(grad N_b . grad A) ]
* conductivity ("mass") matrix, singular because sigma = 0 outside the sheath:
      M_ab = sum_e sigma_e |e| (1 + delta_ab) / 12
* source: uniform impressed current density I(t)/A_core in the stranded core,
      f_a = I(t) / A_core * sum_{e in core, a in e} |e| / 3
  with A_core the discrete core area, so that sum_a f_a = I(t) exactly;
  I(t) = sum_j amp_j sin(2 pi freq_j t + phase_j).

Dirichlet nodes (A = 0 on the outer boundary) are eliminated; vectors below
are over the free nodes only, in node order.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

NU_LINEAR, NU_BRAUER = 0, 1


class FEModel:
    """Assembled FE data of one problem (all FP64)."""

    def __init__(self, problem):
        mesh = problem.mesh
        self.problem = problem
        xy = np.asarray(mesh.xy, dtype=np.float64)
        tri = np.asarray(mesh.tri, dtype=np.int64)
        region = np.asarray(mesh.region, dtype=np.int64)
        free = np.asarray(mesh.dirichlet) == 0
        self.n_nodes = xy.shape[0]
        self.free = free
        self.dof_of_node = np.full(self.n_nodes, -1, dtype=np.int64)
        self.dof_of_node[free] = np.arange(int(free.sum()))
        self.ndof = int(free.sum())

        p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
        det = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])
        if np.any(det == 0.0):
            raise ValueError("degenerate triangle")
        self.area = 0.5 * np.abs(det)
        # grad N_a = (y_b - y_c, x_c - x_b) / det for (a, b, c) cyclic
        grad = np.empty((tri.shape[0], 3, 2))
        grad[:, 0, 0] = (p1[:, 1] - p2[:, 1]) / det
        grad[:, 0, 1] = (p2[:, 0] - p1[:, 0]) / det
        grad[:, 1, 0] = (p2[:, 1] - p0[:, 1]) / det
        grad[:, 1, 1] = (p0[:, 0] - p2[:, 0]) / det
        grad[:, 2, 0] = (p0[:, 1] - p1[:, 1]) / det
        grad[:, 2, 1] = (p1[:, 0] - p0[:, 0]) / det
        self.grad = grad
        self.tri = tri
        self.region = region

        sigma = np.asarray(problem.sigma, dtype=np.float64)[region]
        model = np.asarray(problem.nu_model)[region]
        self.nonlinear = np.nonzero(model == NU_BRAUER)[0]
        self.linear = np.nonzero(model == NU_LINEAR)[0]
        self.nu_lin = np.asarray(problem.nu, dtype=np.float64)[region]
        self.k = np.asarray(problem.brauer, dtype=np.float64)[region]      # (n_tri, 3)
        bmax = np.asarray(getattr(problem, "bmax", np.zeros(len(problem.brauer))), dtype=np.float64)[region]
        self.b2max = np.where(bmax > 0.0, bmax * bmax, np.inf)             # (n_tri,)
        self.sigma = sigma

        # element matrices -> global COO over all nodes, then restrict to free dofs
        ab = np.einsum("eak,ebk->eab", grad, grad)                           # grad N_a . grad N_b
        self._ab = ab
        lin = self.linear
        Klin = self._scatter(lin, self.nu_lin[lin, None, None] * self.area[lin, None, None] * ab[lin])
        cond = np.nonzero(sigma > 0.0)[0]
        mass_loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
        Mloc = sigma[cond, None, None] * self.area[cond, None, None] * mass_loc[None]
        self.K_lin = Klin
        self.M = self._scatter(cond, Mloc)

        src = np.nonzero(np.asarray(problem.is_source)[region] != 0)[0]
        a_core = float(self.area[src].sum())
        g = np.zeros(self.n_nodes)
        np.add.at(g, tri[src].ravel(), np.repeat(self.area[src] / 3.0, 3))
        self.g = g[free] / a_core
        self.a_core = a_core
        self.amp = np.asarray(problem.amp, dtype=np.float64)
        self.freq = np.asarray(problem.freq, dtype=np.float64)
        self.phase = np.asarray(problem.phase, dtype=np.float64)

    # -- assembly helpers -------------------------------------------------
    def _scatter(self, elems, loc):
        """Sum element matrices loc[e, a, b] into a free-dof CSR matrix."""
        t = self.tri[elems]
        rows = np.repeat(t, 3, axis=1).ravel()
        cols = np.tile(t, (1, 3)).ravel()
        vals = loc.reshape(-1)
        dr = self.dof_of_node[rows]
        dc = self.dof_of_node[cols]
        keep = (dr >= 0) & (dc >= 0)
        return sp.csr_matrix((vals[keep], (dr[keep], dc[keep])), shape=(self.ndof, self.ndof))

    def full(self, u):
        """Free-dof vector -> nodal vector with zeros on the Dirichlet boundary."""
        x = np.zeros(self.n_nodes)
        x[self.free] = u
        return x

    def grad_A(self, u, elems):
        """Constant gradient of A on each element in ``elems``: (len, 2)."""
        ue = self.full(u)[self.tri[elems]]                                  # (ne, 3)
        return np.einsum("ea,eak->ek", ue, self.grad[elems])

    def nu_brauer(self, b2, elems):
        k = self.k[elems]
        bc = np.minimum(b2, self.b2max[elems])
        return k[:, 0] * np.exp(k[:, 1] * bc) * (1.0 + k[:, 1] * (b2 - bc)) + k[:, 2]

    def dnu_brauer(self, b2, elems):
        """d nu / d(B^2) (constant past the cap)."""
        k = self.k[elems]
        return k[:, 0] * k[:, 1] * np.exp(k[:, 1] * np.minimum(b2, self.b2max[elems]))

    # -- operators ----------------------------------------------------------
    def Ku(self, u):
        """K(u) u over free dofs."""
        y = self.K_lin @ u
        nl = self.nonlinear
        if nl.size:
            gA = self.grad_A(u, nl)
            b2 = np.einsum("ek,ek->e", gA, gA)
            nu = self.nu_brauer(b2, nl)
            loc = (self.area[nl] * nu)[:, None] * np.einsum("eak,ek->ea", self.grad[nl], gA)
            yn = np.zeros(self.n_nodes)
            np.add.at(yn, self.tri[nl].ravel(), loc.ravel())
            y = y + yn[self.free]
        return y

    def jacobian_K(self, u):
        """d(K(u) u)/du over free dofs (symmetric positive definite)."""
        nl = self.nonlinear
        if nl.size == 0:
            return self.K_lin.copy()
        gA = self.grad_A(u, nl)
        b2 = np.einsum("ek,ek->e", gA, gA)
        nu = self.nu_brauer(b2, nl)
        dnu = self.dnu_brauer(b2, nl)
        s = np.einsum("eak,ek->ea", self.grad[nl], gA)                      # grad N_a . grad A
        loc = self.area[nl, None, None] * (nu[:, None, None] * self._ab[nl]
                                           + 2.0 * dnu[:, None, None] * s[:, :, None] * s[:, None, :])
        return self.K_lin + self._scatter(nl, loc)

    def chord_K(self, u):
        """K(u) itself (the secant matrix, no nu' term)."""
        nl = self.nonlinear
        if nl.size == 0:
            return self.K_lin.copy()
        gA = self.grad_A(u, nl)
        b2 = np.einsum("ek,ek->e", gA, gA)
        nu = self.nu_brauer(b2, nl)
        loc = self.area[nl, None, None] * nu[:, None, None] * self._ab[nl]
        return self.K_lin + self._scatter(nl, loc)

    def current(self, t):
        return float(np.sum(self.amp * np.sin(2.0 * math.pi * self.freq * t + self.phase)))

    def f(self, t):
        return self.current(t) * self.g

    def newton_scale(self):
        """Reference size of the residual: ||g||_2 times the peak current bound."""
        return float(np.linalg.norm(self.g) * np.sum(np.abs(self.amp)))
