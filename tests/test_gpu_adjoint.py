"""Periodic adjoint on the GPU (pppc_adjoint, the autograd wrapper) against the
oracle's adjoint and against central differences of the GPU's own loss."""

import copy
import os

import numpy as np
import pytest

from oracle.adjoint import loss_gradient
from oracle.fem import FEModel
from oracle.periodic import bruteforce_periodic
from synth import REGION_SHEATH, make_problem, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_13076_gb300 import _lib
    from paper_1905_13076_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def mid():
    """A 20 A cable, 181 unknowns, 80 fine levels: the oracle's direct
    periodic and adjoint solves still fit."""
    return make_problem("mid", 10, 20, 8, 10, 5e6, amp=(20.0,))


PROBLEMS = {"tiny": lambda: workload("tiny"), "mid": mid}
_ORACLE = {}


def oracle_reference(name):
    if name not in _ORACLE:
        prob = PROBLEMS[name]()
        m = FEModel(prob)
        traj = bruteforce_periodic(m, prob.N, prob.n_fine, prob.T, tol=1e-12, max_newton=80)
        _ORACLE[name] = loss_gradient(m, traj, prob.T, REGION_SHEATH)
    return _ORACLE[name]


def gpu_adjoint(prob, precision="fp64", tol=1e-12):
    from paper_1905_13076_gb300 import from_problem

    with from_problem(prob, precision=precision, tol_coarse=1e-13) as s:
        s.solve_periodic(tol=tol, kmax=200)
        return s.adjoint(REGION_SHEATH, tol=1e-11)


@pytest.mark.parametrize("name,precision,tol_p,tol_g", [("tiny", "fp64", 1e-9, 1e-7), ("mid", "fp64", 1e-9, 1e-7),
                                                        ("mid", "mixed", 1e-7, 1e-5)])
def test_adjoint_matches_oracle(name, precision, tol_p, tol_g):
    P, g = oracle_reference(name)
    Pg, gg, info = gpu_adjoint(PROBLEMS[name](), precision, tol=1e-12 if precision == "fp64" else 1e-10)
    assert info["rel_res"] <= 1e-11 and info["iterations"] > 0
    assert Pg == pytest.approx(P, rel=tol_p)
    for i in range(4):
        assert gg[i] == pytest.approx(g[i], rel=tol_g), (i, gg[i], g[i])


def _tight_loss(prob, adjoint=False):
    """The GPU's periodic loss solved to its rounding floor (rel_res <= 1e-13,
    Newton 1e-13, PCG 1e-14), so that central differences at h = 1e-6 resolve
    the gradient: with relative sensitivities theta dP/dtheta / P of 0.04 or
    more, a loss error of 1e-14 P costs at most ~1e-7 of the difference."""
    from paper_1905_13076_gb300 import from_problem

    with from_problem(prob, tol_coarse=1e-13, tol_newton=1e-13, tol_lin=1e-14) as s:
        iters, rr = s.solve_periodic(tol=1e-14, kmax=400, raise_on_fail=False)
        assert rr <= 1e-13, rr
        if adjoint:
            return s.adjoint(REGION_SHEATH, tol=1e-12)
        return s.adjoint(REGION_SHEATH, tol=1e-12)[0]


def test_adjoint_gradient_matches_central_differences():
    """dP/d(sigma, k1, k2, k3) of the GPU's own periodic solutions against
    central differences with h = 1e-6 relative, within 1e-6."""
    prob = mid()
    _, grad, _ = _tight_loss(prob, adjoint=True)
    h = 1e-6
    for i, (attr, idx) in enumerate([("sigma", None), ("brauer", 0), ("brauer", 1), ("brauer", 2)]):
        vals = []
        for f in (1 + h, 1 - h):
            p = copy.deepcopy(prob)
            arr = np.array(getattr(p, attr), dtype=np.float64)
            if idx is None:
                arr[REGION_SHEATH] *= f
            else:
                arr[REGION_SHEATH, idx] *= f
            setattr(p, attr, arr)
            vals.append(_tight_loss(p))
        theta = prob.sigma[REGION_SHEATH] if idx is None else prob.brauer[REGION_SHEATH, idx]
        fd = (vals[0] - vals[1]) / (2 * h * theta)
        assert grad[i] == pytest.approx(fd, rel=1e-6), (attr, idx, grad[i], fd)


def test_autograd_function_returns_the_adjoint_gradient():
    import torch

    from paper_1905_13076_gb300.autograd import eddy_loss

    prob = workload("tiny")
    P, g = oracle_reference("tiny")
    theta = torch.tensor([prob.sigma[REGION_SHEATH], *prob.brauer[REGION_SHEATH]], dtype=torch.float64,
                         requires_grad=True)
    loss = eddy_loss(theta, prob, REGION_SHEATH, tol=1e-12, tol_coarse=1e-13)
    (2.0 * loss).backward()
    assert loss.item() == pytest.approx(P, rel=1e-9)
    assert np.allclose(theta.grad.numpy(), 2.0 * g, rtol=1e-7, atol=0)


def test_adjoint_errors():
    from paper_1905_13076_gb300 import PPPCError, from_problem

    prob = workload("tiny")
    with from_problem(prob) as s:
        with pytest.raises(PPPCError) as e:
            s.adjoint(REGION_SHEATH)                 # U = 0 is not the periodic solution
        assert e.value.status == 3
        s.solve_periodic(tol=1e-11)
        with pytest.raises(PPPCError) as e:
            s.adjoint(0)                             # the core is linear and carries no eddy current
        assert e.value.status == 1
