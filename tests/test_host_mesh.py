"""The library's host-side mesh preprocessing (integer work: dof numbering,
CSR pattern, special rows) against the oracle's assembly, bit for bit, on the
CPU.  The library's mesh_host.cpp is compiled here with the host compiler
next to a test-only wrapper (tests/host/mesh_pattern.cpp)."""

import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.fem import FEModel
from synth import REGION_CORE, REGION_SHEATH, workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_13076_gb300", "csrc")
NONLINEAR, CONDUCTIVE, SOURCE = 1, 2, 4


@pytest.fixture(scope="module")
def meshlib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("meshlib") / "libmesh_pattern.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(CSRC, "mesh_host.cpp"), os.path.join(ROOT, "tests", "host", "mesh_pattern.cpp"),
                    "-o", out], check=True)
    lib = ctypes.CDLL(out)
    P, I, PI = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)
    lib.mesh_pattern.restype = I
    lib.mesh_pattern.argtypes = [I, I, P, P, P, I, P, I, PI, PI, P, P, P, P, PI, PI, ctypes.c_char_p, I]
    return lib


def run(meshlib, prob, kinds=None, tri=None):
    m = prob.mesh
    tri = np.ascontiguousarray(m.tri if tri is None else tri, dtype=np.int32)
    reg = np.ascontiguousarray(m.region, dtype=np.int32)
    dir_ = np.ascontiguousarray(m.dirichlet, dtype=np.uint8)
    if kinds is None:
        kinds = np.zeros(4, dtype=np.int32)
        for r in range(4):
            kinds[r] = ((NONLINEAR if prob.nu_model[r] == 1 else 0) | (CONDUCTIVE if prob.sigma[r] > 0 else 0)
                        | (SOURCE if prob.is_source[r] else 0))
    cap = 20 * m.xy.shape[0] + 16
    I = ctypes.c_int
    ndof, nnz, nsp, nnl = I(), I(), I(), I()
    nod, rp, col, rs = (np.zeros(cap, dtype=np.int32) for _ in range(4))
    err = ctypes.create_string_buffer(256)
    st = meshlib.mesh_pattern(m.xy.shape[0], tri.shape[0], tri.ctypes.data, reg.ctypes.data, dir_.ctypes.data, 4,
                              kinds.ctypes.data, cap, ctypes.byref(ndof), ctypes.byref(nnz), nod.ctypes.data,
                              rp.ctypes.data, col.ctypes.data, rs.ctypes.data, ctypes.byref(nsp), ctypes.byref(nnl),
                              err, 256)
    return st, err.value, ndof.value, nnz.value, nod, rp, col, rs, nsp.value, nnl.value


@pytest.mark.parametrize("name", ["tiny", "small", "paper"])
def test_csr_pattern_and_special_rows_match_the_oracle(meshlib, name):
    prob = workload(name)
    om = FEModel(prob)
    st, err, ndof, nnz, nod, rp, col, rs, nsp, nnl = run(meshlib, prob)
    assert st == 0, err
    assert ndof == om.ndof
    assert np.array_equal(nod[:ndof], np.nonzero(om.free)[0])
    # pattern of the full Newton matrix: all element couplings between free dofs
    rng = np.random.default_rng(1)
    u = 1e-3 * rng.standard_normal(om.ndof)
    A = (om.K_lin + om.M + om.jacobian_K(u)).tocsr()
    A.sort_indices()
    # structural pattern (values can cancel): rebuild from the element lists
    rows, cols = [], []
    for t in om.tri:
        d = om.dof_of_node[t]
        for a in d:
            for b in d:
                if a >= 0 and b >= 0:
                    rows.append(a)
                    cols.append(b)
    pat = {(r, c) for r, c in zip(rows, cols)}
    assert nnz == len(pat)
    got = {(i, int(c)) for i in range(ndof) for c in col[rp[i]:rp[i + 1]]}
    assert got == pat
    for i in range(ndof):                                  # columns ascending, diagonal present
        cs = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cs) > 0) and i in cs
    assert set(zip(*A.nonzero())) <= pat
    # special rows: touch a nonlinear or conductive element
    spec = np.zeros(om.ndof, dtype=bool)
    for e in np.nonzero((om.region == REGION_SHEATH))[0]:
        for v in om.tri[e]:
            if om.dof_of_node[v] >= 0:
                spec[om.dof_of_node[v]] = True
    assert np.array_equal(rs[:ndof] >= 0, spec)
    assert nsp == int(spec.sum())
    assert nnl == int(np.sum(om.region == REGION_SHEATH))


def test_invalid_meshes_are_rejected_with_a_message(meshlib):
    prob = workload("tiny")
    tri = prob.mesh.tri.copy()
    tri[3, 1] = tri[3, 0]
    st, err, *_ = run(meshlib, prob, tri=tri)
    assert st == 1 and b"repeats a node" in err
    tri = prob.mesh.tri.copy()
    tri[0, 0] = 10_000
    st, err, *_ = run(meshlib, prob, tri=tri)
    assert st == 1 and b"out of range" in err
    assert REGION_CORE == 0
