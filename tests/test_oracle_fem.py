"""Pins of the oracle's space discretisation (Sec. 2, Eq. 1) against things
other than itself: finite differences, conservation, symmetry and the analytic
skin-effect solution of the continuous problem."""

import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.bessel import coax_phasor
from oracle.fem import FEModel
from synth import NU0, RADII, REGION_SHEATH, coax_mesh, make_problem, workload


@pytest.fixture(scope="module")
def small():
    return FEModel(workload("small"))


def _field_in_knee(model, seed=3):
    """A state whose sheath flux density is around 1-2 T (the Brauer knee)."""
    rng = np.random.default_rng(seed)
    xy = model.problem.mesh.xy[model.free]
    r = np.hypot(xy[:, 0], xy[:, 1])
    u = 1.5 * (RADII[3] - r)                                    # |grad A| ~ 1.5 T
    return u * (1.0 + 0.001 * rng.standard_normal(u.size))


def test_flux_density_reaches_knee(small):
    u = _field_in_knee(small)
    gA = small.grad_A(u, small.nonlinear)
    B = np.sqrt((gA ** 2).sum(1))
    assert 0.5 < np.median(B) < 3.0


def test_jacobian_matches_central_differences(small):
    u = _field_in_knee(small)
    v = np.random.default_rng(7).standard_normal(small.ndof) * 1e-6
    J = small.jacobian_K(u)
    errs = []
    for h in (1.0, 0.1, 0.01):
        fd = (small.Ku(u + h * v) - small.Ku(u - h * v)) / (2 * h)
        errs.append(np.linalg.norm(fd - J @ v) / np.linalg.norm(fd))
    assert errs[2] < 1e-8
    assert errs[1] < errs[0] / 50.0                 # second-order difference error
    # the nu' term matters here: dropping it fails the check
    chord = small.chord_K(u)
    assert np.linalg.norm(fd - chord @ v) > 1e-4 * np.linalg.norm(fd)


def test_dnu_matches_difference_quotient(small):
    el = small.nonlinear[:5]
    b2 = np.linspace(0.1, 3.0, 5)
    h = 1e-6
    fd = (small.nu_brauer(b2 + h, el) - small.nu_brauer(b2 - h, el)) / (2 * h)
    assert np.allclose(fd, small.dnu_brauer(b2, el), rtol=1e-8)
    k1, k2, k3 = small.k[el[0]]
    assert small.nu_brauer(np.array([0.0]), el[:1])[0] == pytest.approx(k1 + k3)


def test_brauer_cap_continues_along_the_tangent(small):
    """Past |B| = bmax the law follows its tangent in b = |B|^2: nu and nu'
    continuous at the cap, nu linear in b beyond it, unchanged below it."""
    el = small.nonlinear[:1]
    k1, k2, k3 = small.k[el[0]]
    bc = small.b2max[el[0]]
    assert bc == pytest.approx(9.0)                           # 3 T in the sheath of the workloads
    nu_c = k1 * math.exp(k2 * bc) + k3
    d_c = k1 * k2 * math.exp(k2 * bc)
    eps = 1e-9 * bc
    lo = small.nu_brauer(np.array([bc - eps]), el)[0]
    hi = small.nu_brauer(np.array([bc + eps]), el)[0]
    assert lo == pytest.approx(nu_c, rel=1e-7) and hi == pytest.approx(nu_c, rel=1e-7)
    assert small.dnu_brauer(np.array([bc - eps]), el)[0] == pytest.approx(d_c, rel=1e-7)
    assert small.dnu_brauer(np.array([bc + eps, 4 * bc]), el) == pytest.approx([d_c, d_c], rel=1e-12)
    far = np.array([2 * bc, 10 * bc])
    assert small.nu_brauer(far, el[[0, 0]]) == pytest.approx(nu_c + d_c * (far - bc), rel=1e-12)
    b2 = np.array([0.5, 4.0])
    assert np.allclose(small.nu_brauer(b2, el[[0, 0]]), k1 * np.exp(k2 * b2) + k3, rtol=1e-14)
    # the difference quotient of nu matches nu' on both sides of the cap
    h = 1e-6
    for b in (bc - 0.5, bc + 0.5):
        fd = (small.nu_brauer(np.array([b + h]), el) - small.nu_brauer(np.array([b - h]), el)) / (2 * h)
        assert fd[0] == pytest.approx(small.dnu_brauer(np.array([b]), el)[0], rel=1e-6)


def test_jacobian_matches_central_differences_above_the_cap(small):
    """A 4 T field: every sheath element is past the cap."""
    xy = small.problem.mesh.xy[small.free]
    r = np.hypot(xy[:, 0], xy[:, 1])
    u = 4.0 * (RADII[3] - r) * (1.0 + 0.001 * np.random.default_rng(5).standard_normal(r.size))
    gA = small.grad_A(u, small.nonlinear)
    assert np.all((gA ** 2).sum(1) > small.b2max[small.nonlinear])
    v = np.random.default_rng(8).standard_normal(small.ndof) * 1e-6
    J = small.jacobian_K(u)
    h = 0.01
    fd = (small.Ku(u + h * v) - small.Ku(u - h * v)) / (2 * h)
    assert np.linalg.norm(fd - J @ v) < 1e-8 * np.linalg.norm(fd)
    assert np.linalg.norm(fd - small.chord_K(u) @ v) > 1e-4 * np.linalg.norm(fd)   # the nu' term is kept


def test_matrices_symmetric_and_definite(small):
    u = _field_in_knee(small)
    for A in (small.K_lin, small.M, small.jacobian_K(u)):
        assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    J = (small.M / 1e-5 + small.jacobian_K(u)).toarray()
    np.linalg.cholesky(J)                     # SPD


def test_mass_integrates_conductivity(small):
    mesh = small.problem.mesh
    sheath = np.nonzero(mesh.region == REGION_SHEATH)[0]
    sigma = small.problem.sigma[REGION_SHEATH]
    assert small.M.sum() == pytest.approx(sigma * small.area[sheath].sum(), rel=1e-13)
    # the annulus area is approached from below by the inscribed polygon rings
    annulus = math.pi * (RADII[2] ** 2 - RADII[1] ** 2)
    assert 0.98 * annulus < small.area[sheath].sum() < annulus


def test_source_carries_the_total_current(small):
    for t in (0.0013, 0.005, 0.0171):
        assert small.f(t).sum() == pytest.approx(small.current(t), rel=1e-13, abs=1e-15)
    assert small.current(0.005) == pytest.approx(10.0, rel=1e-12)      # 10 A peak at T/4


def _fe_phasor_error(nr, nth):
    prob = make_problem("bessel", nr, nth, 4, 1, 5e6, linear_sheath=True, jitter=0.0)
    m = FEModel(prob)
    w = 2 * math.pi * 50.0
    A = (m.K_lin + 1j * w * m.M).astype(np.complex128).tocsc()
    Ah = spla.splu(A).solve(10.0 * m.g.astype(np.complex128))
    xy = prob.mesh.xy[m.free]
    exact = coax_phasor(np.hypot(xy[:, 0], xy[:, 1]), 10.0, 50.0, 5e6, prob.nu[REGION_SHEATH], NU0, RADII)
    return np.abs(Ah - exact).max() / np.abs(exact).max()


def test_skin_effect_closed_form_second_order():
    """FE phasor solution vs the Bessel-function solution of the continuous
    linear problem: small error, shrinking about 4x per mesh halving."""
    e1 = _fe_phasor_error(20, 40)
    e2 = _fe_phasor_error(40, 80)
    e3 = _fe_phasor_error(80, 160)
    assert e1 < 2e-3
    assert e3 < e2 / 3.0
    assert e3 < 2.5e-4


def test_closed_form_satisfies_interface_conditions():
    """The analytic solution itself: A continuous, nu A' continuous, A(R4) = 0,
    and the field outside the sheath carries the enclosed current."""
    nu_s = 400.0
    A = lambda r: coax_phasor(np.atleast_1d(r), 10.0, 50.0, 5e6, nu_s, NU0, RADII)
    h = 1e-8
    for R, nl, nr_ in ((RADII[0], NU0, NU0), (RADII[1], NU0, nu_s), (RADII[2], nu_s, NU0)):
        dl = (A(R - h)[0] - A(R - 3 * h)[0]) / (2 * h)
        dr = (A(R + 3 * h)[0] - A(R + h)[0]) / (2 * h)
        left = A(R - h)[0] + h * dl                 # one-sided extrapolations to R
        right = A(R + h)[0] - h * dr
        assert abs(left - right) <= 1e-6 * abs(left)
        assert abs(nl * dl - nr_ * dr) <= 1e-3 * abs(nl * dl)
    assert abs(A(RADII[3])[0]) <= 1e-12 * abs(A(RADII[0])[0])
    # Ampere: in the insulation nu0 * 2 pi r A' = -I
    r = 1.5e-3
    d = (A(r + h)[0] - A(r - h)[0]) / (2 * h)
    assert NU0 * 2 * math.pi * r * d == pytest.approx(-10.0, rel=1e-5)


def test_mesh_fixture_counts():
    m = coax_mesh(20, 40)
    assert m.ndof == 1 + 19 * 40
    assert m.n_tri == 40 + 2 * 40 * 19
    p = m.xy[m.tri]
    det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    assert (det > 0).all()
    assert coax_mesh(28, 84).ndof == 2269                   # the paper's DOF count (Sec. 4)
    a = coax_mesh(20, 40, seed=5)
    b = coax_mesh(20, 40, seed=5)
    assert np.array_equal(a.xy, b.xy)
