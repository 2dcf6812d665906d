"""The library's host multigrid setup (csrc/amg_host.cpp, the fine PCG's
preconditioner with pppc_config.precond = 2), compiled here with the host
compiler next to a test-only wrapper (tests/host/amg_wrapper.cpp), against
SciPy on the oracle's matrices: every coarse matrix is the Galerkin product
P^T A P, the restriction is P^T, and the tables that rebuild a lane's coarse
matrices from its own fine Jacobian reproduce P^T J P at every level.  A
NumPy V-cycle made of the same pieces (l1-Jacobi smoothing) is an SPD
preconditioner whose PCG iteration count does not grow with the mesh."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import FEModel
from synth import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_13076_gb300", "csrc")


@pytest.fixture(scope="module")
def amglib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("amglib") / "libamg.so")
    subprocess.run([cxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", CSRC, os.path.join(CSRC, "amg_host.cpp"),
                    os.path.join(ROOT, "tests", "host", "amg_wrapper.cpp"), "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.amg_build.restype = I
    lib.amg_build.argtypes = [I, P, P, P, P, I]
    lib.amg_field.restype = I
    lib.amg_field.argtypes = [I, ctypes.c_char_p, P, I]
    lib.amg_error.restype = ctypes.c_char_p
    return lib


def field(lib, level, name, dtype):
    n = lib.amg_field(level, name.encode(), None, 0)
    a = np.zeros(max(n, 0), dtype=dtype)
    if n > 0:
        assert lib.amg_field(level, name.encode(), a.ctypes.data, n) == n
    return a


def problem(name):
    """Representative matrix A0 = J(0) + M/dt, a lane's Jacobian J(u) + M/dt at
    a sheath flux density of about 1.5 T, both on one sorted pattern, and the
    special rows (those touching the conducting, nonlinear sheath)."""
    prob = workload(name)
    m = FEModel(prob)
    dt = prob.T / (prob.N * prob.n_fine)
    xy = prob.mesh.xy[m.free]
    u = 0.75 * (4e-3 - np.hypot(xy[:, 0], xy[:, 1]))          # |grad u| = 0.75 T
    u *= 2.0
    A0 = (m.jacobian_K(np.zeros(m.ndof)) + m.M / dt).tocsr()
    J = (m.jacobian_K(u) + m.M / dt).tocsr()
    S = (abs(A0) + abs(J)).tocsr()
    S.sort_indices()
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    a0 = np.asarray(A0[rows, S.indices]).ravel()
    jv = np.asarray(J[rows, S.indices]).ravel()
    special = np.asarray(abs(m.M).sum(axis=1)).ravel() > 0
    row_slot = np.full(S.shape[0], -1, dtype=np.int32)
    lens = np.diff(S.indptr)
    row_slot[special] = np.concatenate([[0], np.cumsum(lens[special])[:-1]]).astype(np.int32)
    pat = (S.indptr.astype(np.int32), S.indices.astype(np.int32))
    return pat, a0, jv, row_slot, special


def build(lib, pat, a0, row_slot, coarse_rows=400):
    rowptr, col = pat
    nl = lib.amg_build(len(rowptr) - 1, rowptr.ctypes.data, col.ctypes.data, a0.ctypes.data, row_slot.ctypes.data,
                       coarse_rows)
    assert nl > 0, lib.amg_error()
    levels = []
    for l in range(nl):
        L = {k: field(lib, l, k, np.int32) for k in ("rowptr", "col", "row_slot", "sp_index", "Pptr", "Pcol",
                                                      "Rptr", "Rcol", "cptr", "csrc")}
        L.update({k: field(lib, l, k, np.float64) for k in ("val", "l1", "Pval", "Rval", "slot_base", "cw")})
        L["cost"] = field(lib, l, "cost", np.int64)
        n = len(L["rowptr"]) - 1
        L["A"] = sp.csr_matrix((L["val"], L["col"], L["rowptr"]), shape=(n, n))
        if l > 0:
            nf = len(levels[-1]["rowptr"]) - 1
            L["P"] = sp.csr_matrix((L["Pval"], L["Pcol"], L["Pptr"]), shape=(nf, n))
            L["R"] = sp.csr_matrix((L["Rval"], L["Rcol"], L["Rptr"]), shape=(n, nf))
        levels.append(L)
    return levels


def lane_matrices(levels, jv):
    """Each level's matrix for one lane: shared rows from the representative
    values, special rows from the lane's slots, rebuilt with the tables."""
    L0 = levels[0]
    sp0 = L0["row_slot"] >= 0
    k0 = np.repeat(sp0, np.diff(L0["rowptr"]))
    # level 0 slots: the lane's special-row entries, at their slot numbers
    rows = np.repeat(np.arange(len(sp0)), np.diff(L0["rowptr"]))[k0]
    kk = np.nonzero(k0)[0]
    slots = np.empty(int(k0.sum()))
    slots[L0["row_slot"][rows] + (kk - L0["rowptr"][rows])] = jv[k0]
    mats = [sp.csr_matrix((np.where(k0, jv, L0["val"]), L0["col"], L0["rowptr"]), shape=L0["A"].shape)]
    for L in levels[1:]:
        owner = np.repeat(np.arange(len(L["slot_base"])), np.diff(L["cptr"]))
        slots = L["slot_base"] + np.bincount(owner, weights=L["cw"] * slots[L["csrc"]],
                                             minlength=len(L["slot_base"]))
        k = np.repeat(L["row_slot"] >= 0, np.diff(L["rowptr"]))
        vals = L["val"].copy()
        vals[k] = slots
        mats.append(sp.csr_matrix((vals, L["col"], L["rowptr"]), shape=L["A"].shape))
    return mats


def rel(a, b):
    return abs(a - b).max() / abs(b).max()


@pytest.fixture(scope="module")
def small(amglib):
    pat, a0, jv, row_slot, special = problem("small")
    return pat, a0, jv, row_slot, special, build(amglib, pat, a0, row_slot, coarse_rows=40)


def test_hierarchy_is_galerkin(small):
    pat, a0, jv, row_slot, special, levels = small
    assert len(levels) >= 3
    sizes = [L["A"].shape[0] for L in levels]
    assert all(b < 0.85 * a for a, b in zip(sizes, sizes[1:]))
    for f, c in zip(levels, levels[1:]):
        assert rel(c["A"], (c["P"].T @ f["A"] @ c["P"]).tocsr()) < 1e-12
        assert abs(c["R"] - c["P"].T).max() == 0
        # smoothed prolongator: every fine row reaches some aggregate
        assert (np.diff(c["Pptr"]) > 0).all()
        np.testing.assert_allclose(c["l1"], np.asarray(abs(c["A"]).sum(axis=1)).ravel(), rtol=1e-12)


def test_lane_tables_rebuild_the_lane_galerkin_products(small):
    """For a lane whose fine Jacobian differs from the representative matrix
    on the special rows, the tabulated slots give P^T J P at every level,
    and the coarse rows outside the tables keep the shared values."""
    pat, a0, jv, row_slot, special, levels = small
    assert rel(jv, a0) > 1e-3                             # the lane is far from the representative matrix
    mats = lane_matrices(levels, jv)
    for l in range(1, len(levels)):
        P = levels[l]["P"]
        ref = (P.T @ mats[l - 1] @ P).tocsr()
        assert rel(mats[l], ref) < 1e-12, l
        # the per-lane rows are exactly those a per-lane finer row prolongs into
        fine_sp = levels[l - 1]["row_slot"] >= 0
        reach = np.asarray(abs(P[fine_sp]).sum(axis=0)).ravel() > 0
        assert ((levels[l]["row_slot"] >= 0) == reach).all()


def test_work_prefix_counts_each_rows_vcycle_work(small):
    """Every coarse level carries the prefix of its rows' V-cycle work, the
    key of the split of its rows among a team's blocks: two residual passes
    (twice the reads on a special row), the restriction row, the row of the
    next level's prolongation, and 4 per row."""
    levels = small[-1]
    assert len(levels[0]["cost"]) == 0
    for l in range(1, len(levels)):
        L = levels[l]
        nnz_a = np.diff(L["rowptr"])
        w = 2 * nnz_a * (1 + (L["row_slot"] >= 0)) + np.diff(L["Rptr"]) + 4
        if l + 1 < len(levels):
            w = w + np.diff(levels[l + 1]["Pptr"])
        assert L["cost"][0] == 0 and len(L["cost"]) == len(nnz_a) + 1
        np.testing.assert_array_equal(np.diff(L["cost"]), w)
        assert (np.diff(L["cost"]) > 0).all()


def test_tables_do_not_depend_on_the_fine_slot_order(amglib):
    """With the fine special rows' slots numbered in reverse row order (every
    coarse slot's contributions then arrive out of order and are sorted), the
    tables still rebuild P^T J P at every level."""
    pat, a0, jv, row_slot, special = problem("small")
    lens = np.diff(pat[0])
    rs = np.full(len(lens), -1, dtype=np.int32)
    rows = np.nonzero(special)[0][::-1]
    rs[rows] = np.concatenate([[0], np.cumsum(lens[rows])[:-1]]).astype(np.int32)
    levels = build(amglib, pat, a0, rs, coarse_rows=40)
    assert len(levels) >= 3
    mats = lane_matrices(levels, jv)
    for l in range(1, len(levels)):
        P = levels[l]["P"]
        assert rel(mats[l], (P.T @ mats[l - 1] @ P).tocsr()) < 1e-12, l
        cptr, csrc = levels[l]["cptr"], levels[l]["csrc"]
        for e in range(len(cptr) - 1):                   # sorted, merged per coarse slot
            assert (np.diff(csrc[cptr[e]:cptr[e + 1]]) > 0).all()


def vcycle(levels, mats, r, sweeps=2):
    l1 = [np.asarray(abs(A).sum(axis=1)).ravel() for A in mats]

    def down_up(l, b):
        A = mats[l]
        y = b / l1[l]
        if l == len(levels) - 1:
            for _ in range(sweeps - 1):
                y = y + (b - A @ y) / l1[l]
            return y
        P = levels[l + 1]["P"]
        y = y + P @ down_up(l + 1, levels[l + 1]["R"] @ (b - A @ y))
        return y + (b - A @ y) / l1[l]

    return down_up(0, r)


def pcg_iterations(A, b, prec, tol):
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = r @ z
    for k in range(3000):
        if np.linalg.norm(r) <= tol * np.linalg.norm(b):
            return k
        w = A @ p
        den = p @ w
        assert den > 0                                    # SPD preconditioned operator: no breakdown
        a = rz / den
        x += a * p
        r -= a * w
        z = prec(r)
        rz2 = r @ z
        p = z + rz2 / rz * p
        rz = rz2
    return 3000


def test_vcycle_is_symmetric_positive_definite(small):
    """The V-cycle built from a lane's own matrices (l1-Jacobi smoothing,
    R = P^T, a symmetric coarsest sweep) is a symmetric positive definite
    operator: its matrix, probed column by column, is symmetric with
    positive eigenvalues."""
    pat, a0, jv, row_slot, special, levels = small
    mats = lane_matrices(levels, jv)
    n = mats[0].shape[0]
    B = np.column_stack([vcycle(levels, mats, e) for e in np.eye(n)])
    assert np.abs(B - B.T).max() <= 1e-10 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@pytest.mark.parametrize("name,max_its,gain", [("small", 30, 2), ("medium", 45, 8)])
def test_vcycle_pcg_iterations_stay_low(amglib, name, max_its, gain):
    """PCG on a lane's Jacobian with the V-cycle needs few iterations on both
    meshes; Jacobi-PCG needs many more, and more on the finer mesh."""
    pat, a0, jv, row_slot, special = problem(name)
    levels = build(amglib, pat, a0, row_slot)
    mats = lane_matrices(levels, jv)
    J = mats[0]
    b = np.random.default_rng(3).standard_normal(J.shape[0])
    k_amg = pcg_iterations(J, b, lambda r: vcycle(levels, mats, r), 1e-4)
    d = J.diagonal()
    k_jac = pcg_iterations(J, b, lambda r: r / d, 1e-4)
    assert k_amg <= max_its, (k_amg, k_jac)
    assert gain * k_amg < k_jac
