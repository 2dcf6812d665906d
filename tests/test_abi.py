"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/pppc.h.  Host-only calls (no GPU needed) are exercised."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pppc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pppc_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_13076_gb300 import _lib
    from paper_1905_13076_gb300 import build as b

    if not os.path.exists(_lib.LIB_PATH):
        b.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pppc_create", "pppc_set_mesh", "pppc_iterate", "pppc_solve_periodic",
              "pppc_propagate_fine", "pppc_coarse_update", "pppc_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1905_13076_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pppc_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the binding declares exactly those
    assert set(_lib.SIGNATURES) == set(declared_functions())


def test_build_targets_sm103a_only():
    """Every translation unit and the link use one -gencode for sm_103a; the
    loaded library's kernels report that target on a GPU
    (test_gpu_parity.py::test_kernels_report_sm103)."""
    from paper_1905_13076_gb300 import build as b

    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_config_defaults_and_validation(lib):
    from paper_1905_13076_gb300._lib import pppc_config

    cfg = pppc_config()
    lib.pppc_config_default(ctypes.byref(cfg))
    assert cfg.T == 0.02 and cfg.N == 16 and cfg.n_fine == 20 and cfg.tol_newton == 1e-10
    h = ctypes.c_void_p()
    cfg.N = 15                                   # odd N: no Hermitian spectrum split
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None
    assert b"even" in lib.pppc_last_error(None)
    cfg.N = 16
    cfg.T = -1.0
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.T = 0.02
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    assert h.value
    # calls out of order are refused before any device work
    rr = ctypes.c_double()
    assert lib.pppc_iterate(h, ctypes.byref(rr)) == 3
    assert lib.pppc_ndof(h) == 0
    lib.pppc_destroy(h)
    assert lib.pppc_status_string(9) == b"PPPC_ERR_NOT_CONVERGED"


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_1905_13076_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_config_options_are_validated(lib):
    """Every option field of pppc_config is range-checked at create time (no
    device work): method, coarse_at, newton_schedule, precond, predictor."""
    from paper_1905_13076_gb300._lib import pppc_config

    cases = [("method", 2, b"method"), ("coarse_at", 2, b"coarse_at"), ("newton_schedule", 2, b"newton_schedule"),
             ("precond", 3, b"precond"), ("predictor", 3, b"predictor"), ("precision", 5, b"precision"),
             ("coarse_lin", 7, b"coarse_lin"), ("eta0", 1.5, b"eta0")]
    for field, bad, word in cases:
        cfg = pppc_config()
        lib.pppc_config_default(ctypes.byref(cfg))
        setattr(cfg, field, bad)
        h = ctypes.c_void_p()
        assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 1, field
        assert h.value is None
        assert word in lib.pppc_last_error(None), (field, lib.pppc_last_error(None))
    cfg = pppc_config()
    lib.pppc_config_default(ctypes.byref(cfg))
    assert (cfg.method, cfg.coarse_at, cfg.newton_schedule, cfg.precond, cfg.predictor) == (0, 0, 0, 0, 1)
    for field, good in [("method", 1), ("coarse_at", 1), ("newton_schedule", 1), ("precond", 1), ("predictor", 2)]:
        c2 = pppc_config()
        lib.pppc_config_default(ctypes.byref(c2))
        setattr(c2, field, good)
        h = ctypes.c_void_p()
        assert lib.pppc_create(ctypes.byref(c2), ctypes.byref(h)) == 0, field
        lib.pppc_destroy(h)


def test_batch_and_adjoint_refuse_bad_arguments_without_a_device(lib):
    """Argument checks of the batch and adjoint calls come before any device work."""
    from paper_1905_13076_gb300._lib import pppc_adjoint_result, pppc_config

    b = ctypes.c_void_p()
    assert lib.pppc_batch_create(None, 0, 1, ctypes.byref(b)) == 1
    assert b"count" in lib.pppc_batch_last_error(None)
    cfg = pppc_config()
    lib.pppc_config_default(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    arr = (ctypes.c_void_p * 1)(h.value)
    assert lib.pppc_batch_create(arr, 1, 1, ctypes.byref(b)) == 3        # member without a mesh
    arr2 = (ctypes.c_void_p * 2)(h.value, h.value)
    assert lib.pppc_batch_create(arr2, 2, 1, ctypes.byref(b)) == 1       # the same member twice
    res = pppc_adjoint_result()
    assert lib.pppc_adjoint(h, 2, 1e-10, 10, ctypes.byref(res)) == 3     # no mesh yet
    lib.pppc_destroy(h)


def test_batch_plan_minimises_the_slowest_team(lib):
    """The tuner's greedy split equals the brute-force optimum of
    max cost / blocks on small cases, respects caps and skips inactive
    members (host-only call)."""
    import itertools

    import numpy as np

    D, I = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    rng = np.random.default_rng(4)
    for trial in range(60):
        n = int(rng.integers(1, 5))
        total = int(rng.integers(n, 9))
        cost = rng.uniform(0.1, 10.0, n)
        cap = rng.integers(1, 6, n).astype(np.int32)
        active = (rng.uniform(size=n) < 0.8).astype(np.int32)
        if not active.any():
            active[0] = 1
        blocks = np.zeros(n, dtype=np.int32)
        mk = ctypes.c_double()
        st = lib.pppc_batch_plan(cost.ctypes.data_as(D), cap.ctypes.data_as(I), active.ctypes.data_as(I), n, total,
                                 blocks.ctypes.data_as(I), ctypes.byref(mk))
        assert st == 0
        act = active.astype(bool)
        assert np.all(blocks[~act] == 0) and np.all(blocks[act] >= 1) and np.all(blocks <= np.maximum(cap, 0))
        assert blocks.sum() <= total
        best = np.inf
        idx = np.nonzero(act)[0]
        for combo in itertools.product(*[range(1, int(cap[i]) + 1) for i in idx]):
            if sum(combo) <= total:
                best = min(best, max(cost[i] / b for i, b in zip(idx, combo)))
        assert mk.value == pytest.approx(best, rel=1e-12), (trial, blocks, mk.value, best)
    one = np.ones(2, dtype=np.int32)
    assert lib.pppc_batch_plan(np.ones(2).ctypes.data_as(D), one.ctypes.data_as(I), one.ctypes.data_as(I), 2, 1,
                               np.zeros(2, dtype=np.int32).ctypes.data_as(I), None) == 1   # fewer blocks than members


def test_invalid_meshes_are_refused_before_device_work(lib):
    """set_mesh validates indices, regions, materials and the source on the
    host: each of these inputs is refused with INVALID_ARG (no GPU needed)."""
    import numpy as np

    from paper_1905_13076_gb300._lib import pppc_config, pppc_material

    cfg = pppc_config()
    lib.pppc_config_default(ctypes.byref(cfg))
    h = ctypes.c_void_p()
    assert lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    xy = np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.float64)
    tri = np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32)
    region = np.array([0, 0], dtype=np.int32)
    dirichlet = np.array([0, 0, 0, 1], dtype=np.uint8)
    mats = (pppc_material * 1)()
    mats[0].nu_model, mats[0].nu, mats[0].is_source = 0, 1.0, 1

    def set_mesh(t=tri, reg=region, m=mats, nreg=1):
        return lib.pppc_set_mesh(h, 4, xy.ctypes.data, t.shape[0], t.ctypes.data, reg.ctypes.data,
                                 dirichlet.ctypes.data, nreg, m)

    bad_tri = tri.copy()
    bad_tri[1, 2] = 7                                         # node index out of range
    assert set_mesh(t=bad_tri) == 1
    bad_reg = np.array([0, 3], dtype=np.int32)                # region index out of range
    assert set_mesh(reg=bad_reg) == 1
    m2 = (pppc_material * 1)()
    m2[0].nu_model, m2[0].nu, m2[0].is_source = 0, -1.0, 1    # negative reluctivity
    assert set_mesh(m=m2) == 1
    m3 = (pppc_material * 1)()
    m3[0].nu_model, m3[0].nu, m3[0].is_source = 0, 1.0, 0     # no source region
    assert set_mesh(m=m3) == 1
    m4 = (pppc_material * 1)()
    m4[0].nu_model, m4[0].k1, m4[0].k2, m4[0].k3, m4[0].bmax, m4[0].is_source = 1, 3.8, 2.17, 396.2, -1.0, 1
    assert set_mesh(m=m4) == 1                                # negative Brauer cap
    assert lib.pppc_ndof(h) == 0                              # nothing was set up
    lib.pppc_destroy(h)


def test_python_layer_raises_the_library_status(lib):
    """The binding marshals arguments only: an error status of the C call
    comes back as PPPCError with that status and the library's message."""
    from paper_1905_13076_gb300 import PPPC, PPPCBatch, PPPCError

    s = PPPC(0.02, 16, 20)                              # creating a handle needs no device
    with pytest.raises(PPPCError) as e:
        s.iterate()
    assert e.value.status == 3 and "set_mesh" in e.value.message
    with pytest.raises(PPPCError) as e:
        s.adjoint(2)
    assert e.value.status == 3
    with pytest.raises(PPPCError) as e:
        PPPCBatch([s])
    assert e.value.status == 3 and "member 0" in e.value.message
    with pytest.raises(PPPCError) as e:
        PPPC(0.02, 15, 20)                              # odd N
    assert e.value.status == 1
    with pytest.raises(KeyError):
        PPPC(0.02, 16, 20, precond="ilu")               # unknown option names fail in Python
    s.close()
