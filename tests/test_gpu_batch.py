"""Batched many-problem PP-PC (pppc_batch_*) against single handles and the oracle.

A batch runs every member's fine sweep on its own team of blocks inside one
cooperative launch, and all members' harmonic solves in another, from two
captured CUDA graphs per iteration.  Each member's result must match what
the same member gives alone (the only difference is the order of the
cross-block sums) and, for the small members, the FP64 oracle.
"""

import os

import numpy as np
import pytest

from oracle.fem import FEModel
from oracle.pppc import pppc as oracle_pppc
from synth import make_problem

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL_MIXED = 1e-7


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def uneven_cables():
    """Four cables of different mesh, N, n_fine, sheath sigma and current."""
    return [
        make_problem("c0", 12, 24, 16, 10, 5e6, amp=(10.0,), seed=1),
        make_problem("c1", 8, 16, 32, 6, 2e7, amp=(30.0,), seed=2),
        make_problem("c2", 16, 32, 16, 8, 1e6, amp=(3.0,), seed=3),
        make_problem("c3", 5, 8, 4, 3, 5e6, amp=(10.0,), seed=4),
    ]


def members(problems, **cfg):
    from paper_1905_13076_gb300 import from_problem

    return [from_problem(p, **cfg) for p in problems]


def close_all(ms):
    for m in ms:
        m.close()


def test_batch_solve_matches_single_handles_and_oracle():
    from paper_1905_13076_gb300 import PPPCBatch

    probs = uneven_cables()
    solo = []
    for p in probs:
        with members([p], tol_coarse=1e-12)[0] as s:
            it, rr = s.solve_periodic(tol=1e-11, kmax=40)
            solo.append((it, rr, s.get_state()))
    ms = members(probs, tol_coarse=1e-12)
    with PPPCBatch(ms) as b:
        its, rrs = b.solve_periodic(tol=1e-11, kmax=40)
        st = b.stats()
        fb, cb = b.teams()
    for c, p in enumerate(probs):
        it, rr, U = solo[c]
        assert rrs[c] <= 1e-11
        assert abs(int(its[c]) - it) <= 1, (c, its[c], it)
        assert rel(ms[c].get_state(), U) < TOL64, c
    # the two smallest members against the oracle
    for c in (1, 3):
        p = probs[c]
        ref = oracle_pppc(FEModel(p), p.N, p.n_fine, p.T, tol=1e-11, kmax=40)
        assert ref.converged
        assert rel(ms[c].get_state()[:, p.mesh.dirichlet == 0], ref.U) < TOL64, c
    assert st["iterations"] == int(its.max()) + 1
    assert st["graph_launches"] == 2 * int(its.max()) + 1
    assert st["fine_dof_steps"] == sum((int(its[c]) + 1) * p.N * p.n_fine * ms[c].ndof for c, p in enumerate(probs))
    assert st["kernel_launches"] > 0 and st["fine_ms"] > 0 and st["coarse_ms"] > 0
    # teams of the last graphs: only the member(s) still active hold blocks
    assert fb.sum() <= 152 and cb.sum() <= 152
    close_all(ms)


def test_batch_iterate_matches_single_iterate():
    from paper_1905_13076_gb300 import PPPCBatch

    probs = uneven_cables()
    ms = members(probs, tol_coarse=1e-13, tol_lin=1e-12)
    solo = members(probs, tol_coarse=1e-13, tol_lin=1e-12)
    for m, s, p in zip(ms, solo, probs):       # both from rest
        m.set_state(np.zeros((p.N, p.mesh.n_nodes)))
        s.set_state(np.zeros((p.N, p.mesh.n_nodes)))
    with PPPCBatch(ms, autotune=False) as b:
        for k in range(2):
            rr = b.iterate()
            for c, s in enumerate(solo):
                r1 = s.iterate()
                # only the order of the cross-block sums differs; Newton stops at
                # tol 1e-10, so the two agree to about that
                assert rr[c] == pytest.approx(r1, rel=1e-8)
                assert rel(ms[c].get_state(), s.get_state()) < TOL64, (k, c)
        fb, cb = b.teams()
        assert np.all(fb >= 1) and np.all(cb >= 1)
        assert fb.sum() <= 152 and cb.sum() <= 152
        st = b.stats()
        assert st["retunes"] == 0 and st["graph_launches"] == 2
    close_all(ms)
    close_all(solo)


def test_batch_mixed_precision():
    from paper_1905_13076_gb300 import PPPCBatch

    probs = uneven_cables()[:3]
    # Kbar frozen at the fine results: same fixed point as the FP64 reference below
    ms = members(probs, precision="mixed", coarse_at="F")
    with PPPCBatch(ms) as b:
        its, rrs = b.solve_periodic(tol=1e-9, kmax=40)
    for c, p in enumerate(probs):
        with members([p], tol_coarse=1e-12)[0] as s:
            s.solve_periodic(tol=1e-11, kmax=40)
            ref = s.get_state()
        assert rrs[c] <= 1e-9
        assert rel(ms[c].get_state(), ref) < TOL_MIXED, c
    close_all(ms)


def test_batch_rejects_incompatible_members():
    from paper_1905_13076_gb300 import PPPCBatch, PPPCError

    probs = uneven_cables()
    a = members(probs[:1])
    mixed = members(probs[1:2], precision="mixed")
    ppic = members(probs[2:3], method="ppic")
    odd = members([make_problem("odd", 6, 12, 20, 3, 5e6)], precision="mixed")   # 20 lanes / 4 = 5
    for bad, status in (([a[0], mixed[0]], 10), ([a[0], ppic[0]], 10), (odd, 10), ([a[0], a[0]], 1)):
        with pytest.raises(PPPCError) as e:
            PPPCBatch(bad)
        assert e.value.status == status
    close_all(a + mixed + ppic + odd)
