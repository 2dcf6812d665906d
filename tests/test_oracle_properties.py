"""Property checks of the oracle's assembly over random coax meshes (sizes,
seeds, jitter): symmetry and definiteness, conservation of conductivity and
current, the Jacobian against central differences, and the half-wave
antisymmetry of the periodic solution.  A dropped term, a wrong sign or a
transposed element matrix fails them on some mesh, not only on the fixed
fixtures of the other oracle tests."""

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle.fem import FEModel  # noqa: E402
from oracle.periodic import bruteforce_periodic  # noqa: E402
from synth import RADII, make_problem  # noqa: E402

meshes = st.tuples(st.integers(5, 9), st.integers(6, 16), st.integers(0, 10_000),
                   st.floats(0.0, 0.15))


def model_of(params, amp=10.0, N=4, n_fine=3):
    nr, nth, seed, jitter = params
    return FEModel(make_problem("prop", nr, nth, N, n_fine, 5e6, amp=(amp,), seed=seed, jitter=jitter))


def smooth_state(m, peak_tesla, seed):
    rng = np.random.default_rng(seed)
    xy = m.problem.mesh.xy[m.free]
    r = np.hypot(xy[:, 0], xy[:, 1])
    return peak_tesla * (RADII[3] - r) * (1.0 + 0.01 * rng.standard_normal(r.size))


@settings(max_examples=12, deadline=None)
@given(meshes, st.floats(0.1, 2.5))
def test_matrices_are_symmetric_and_the_jacobian_is_definite(params, tesla):
    m = model_of(params)
    u = smooth_state(m, tesla, params[2])
    J = m.jacobian_K(u).toarray()
    K = m.K_lin.toarray()
    M = m.M.toarray()
    for A in (J, K, M):
        assert np.allclose(A, A.T, rtol=0, atol=1e-9 * np.abs(A).max())
    assert np.linalg.eigvalsh(J).min() > 0.0
    assert np.linalg.eigvalsh(M).min() > -1e-12 * np.abs(M).max()


@settings(max_examples=12, deadline=None)
@given(meshes)
def test_conductivity_and_current_are_conserved(params):
    m = model_of(params)
    cond = m.sigma > 0
    # sum of all entries of the consistent mass = sum of sigma |e| over conducting elements
    # whose three vertices are free (Dirichlet rows and columns are eliminated)
    full = np.all(m.free[m.tri], axis=1)
    assert m.M.sum() == pytest.approx(float(np.sum((m.sigma * m.area)[cond & full])), rel=1e-12)
    # the source shape sums to one: f(t) carries exactly I(t)
    assert m.g.sum() == pytest.approx(1.0, rel=1e-12)


@settings(max_examples=10, deadline=None)
@given(meshes, st.floats(0.3, 2.5))
def test_jacobian_matches_central_differences(params, tesla):
    # below the 3 T cap of the Brauer law: there nu is smooth, and central
    # differences are second-order accurate (across the cap the law is only
    # C^1; test_oracle_fem checks a state wholly above it)
    m = model_of(params)
    u = smooth_state(m, tesla, params[2] + 1)
    v = np.random.default_rng(params[2]).standard_normal(m.ndof) * 1e-6
    Jv = m.jacobian_K(u) @ v
    errs = []
    for h in (1e-2, 1e-3):
        fd = (m.Ku(u + h * v) - m.Ku(u - h * v)) / (2 * h)
        errs.append(np.linalg.norm(fd - Jv) / np.linalg.norm(fd))
    # second-order convergence of the difference quotient to J v (coarse
    # jittered meshes reach the steep part of the law, so no fixed h fits all)
    assert errs[1] < 1e-6
    assert errs[1] < errs[0] / 30.0 or errs[1] < 1e-8   # or already at the rounding floor


@settings(max_examples=5, deadline=None)
@given(st.tuples(st.integers(5, 6), st.integers(6, 10), st.integers(0, 10_000), st.floats(0.0, 0.1)))
def test_periodic_solution_is_half_wave_antisymmetric(params):
    """For an odd-harmonic source, u^{m+L/2} = -u^m (K(-u)(-u) = -K(u)u and the
    periodic solution is unique)."""
    m = model_of(params, N=4, n_fine=2)
    prob = m.problem
    traj = bruteforce_periodic(m, prob.N, prob.n_fine, prob.T, tol=1e-11)
    L = traj.shape[0] - 1
    assert np.linalg.norm(traj[L // 2:L] + traj[:L // 2]) <= 1e-8 * np.linalg.norm(traj)


@settings(max_examples=4, deadline=None)
@given(st.integers(5, 6), st.integers(6, 9), st.integers(0, 10_000), st.floats(1e6, 3e7), st.floats(2.0, 30.0))
def test_pppc_fixed_point_is_the_periodic_solution(nr, nth, seed, sigma, amp):
    """On random small cables PP-PC (Eq. 4, multi-harmonic coarse solve)
    converges to the periodic solution found by Newton on all levels at once."""
    from oracle.pppc import pppc

    prob = make_problem("prop", nr, nth, 4, 2, sigma, amp=(amp,), seed=seed)
    m = FEModel(prob)
    ref = bruteforce_periodic(m, prob.N, prob.n_fine, prob.T, tol=1e-12, max_newton=80)
    res = pppc(m, prob.N, prob.n_fine, prob.T, tol=1e-11, kmax=80)
    assert res.converged
    U_ref = ref[0:prob.N * prob.n_fine:prob.n_fine]          # coarse points u^{n n_fine}
    assert np.linalg.norm(res.U - U_ref) <= 1e-8 * np.linalg.norm(U_ref)
