"""Python face of the C ABI: one ``PPPC`` object per problem handle.

States are (N, n_nodes) FP64 arrays: row n is the vector potential at the
coarse point T_n = n T / N (Sec. 2).  Host data may be NumPy arrays; device
data may be torch CUDA tensors, passed by pointer together with the caller's
current stream.  PyTorch only supplies device memory and streams here.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import (COARSE_LIN, NU_BRAUER, NU_LINEAR, PPPC_FP64, PPPC_MIXED, check, pppc_config,
                   pppc_material, pppc_stats)


@dataclass
class Material:
    sigma: float = 0.0
    nu: float = 0.0
    brauer: tuple | None = None   # (k1, k2, k3) for nu(B^2) = k1 exp(k2 B^2) + k3
    is_source: bool = False
    bmax: float = 0.0             # Brauer: |B| past which nu continues linearly in B^2 (0: no cap)


def _as_host(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _torch_allocator(stream):
    """Device-memory callbacks (pppc_config.alloc / free_fn) that take the
    handle's workspace from PyTorch's caching allocator on the handle's
    stream, so it shows in torch.cuda.memory_allocated() and is reused by
    PyTorch after the handle is destroyed.  None when PyTorch has no GPU."""
    try:
        import torch
    except ImportError:
        return None
    if not torch.cuda.is_available():
        return None
    dev = torch.cuda.current_device()
    st = stream if stream is None or isinstance(stream, int) else stream.cuda_stream

    def alloc(nbytes, ctx):
        try:
            s = torch.cuda.ExternalStream(st, device=dev) if st else torch.cuda.default_stream(dev)
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, s)
        except Exception:
            return None                      # the library reports PPPC_ERR_NOMEM

    def free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass                             # interpreter shutdown

    return _lib.ALLOC_FN(alloc), _lib.FREE_FN(free)


class PPPC:
    """Periodic Parareal with periodic coarse problem and multi-harmonic
    coarse solve on one GPU."""

    def __init__(self, T: float, N: int, n_fine: int, precision: str = "fp64",
                 coarse_lin: str = "avg_jacobian", tol_newton: float = 1e-10, max_newton: int = 30,
                 tol_lin: float = 1e-6, max_lin: int = 20000, tol_coarse: float = 1e-8,
                 max_coarse: int = 20000, eta0: float = 1e-2, predictor: int = 1, method: str = "pppc",
                 coarse_at: str = "U", newton_schedule: bool = False, precond: str = "jacobi",
                 lane_team: int = 0, stream=None, torch_memory: bool = True):
        self._lib = _lib.load()
        cfg = pppc_config()
        self._lib.pppc_config_default(ctypes.byref(cfg))
        cfg.T, cfg.N, cfg.n_fine = float(T), int(N), int(n_fine)
        cfg.precision = {"fp64": PPPC_FP64, "mixed": PPPC_MIXED}[precision]
        cfg.coarse_lin = COARSE_LIN[coarse_lin]
        cfg.tol_newton, cfg.max_newton = float(tol_newton), int(max_newton)
        cfg.tol_lin, cfg.max_lin = float(tol_lin), int(max_lin)
        cfg.tol_coarse, cfg.max_coarse = float(tol_coarse), int(max_coarse)
        cfg.eta0, cfg.predictor = float(eta0), int(predictor)
        cfg.method = _lib.METHODS[method]
        cfg.coarse_at = _lib.COARSE_AT[coarse_at]
        cfg.newton_schedule = int(bool(newton_schedule))
        cfg.precond = {"jacobi": 0, "tridiag": 1, "amg": 2}[precond]
        cfg.lane_team = int(lane_team)
        cfg.stream = stream if stream is None or isinstance(stream, int) else stream.cuda_stream
        # device memory from PyTorch's caching allocator (kept alive with the handle)
        self._alloc = _torch_allocator(stream) if torch_memory else None
        if self._alloc is not None:
            cfg.alloc = ctypes.cast(self._alloc[0], ctypes.c_void_p)
            cfg.free_fn = ctypes.cast(self._alloc[1], ctypes.c_void_p)
        self.cfg = cfg
        h = ctypes.c_void_p()
        check(self._lib.pppc_create(ctypes.byref(cfg), ctypes.byref(h)), None)
        self._h = h
        self.N = int(N)
        self.n_nodes = 0

    # -- lifecycle -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pppc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, status):
        check(status, self._h)

    # -- problem definition ------------------------------------------------------
    def set_mesh(self, xy, tri, region, dirichlet, materials):
        xy = _as_host(xy, np.float64)
        tri = _as_host(tri, np.int32)
        region = _as_host(region, np.int32)
        dirichlet = _as_host(dirichlet, np.uint8)
        mats = (pppc_material * len(materials))()
        for r, m in enumerate(materials):
            mats[r].sigma = float(m.sigma)
            mats[r].is_source = int(bool(m.is_source))
            if m.brauer is not None:
                mats[r].nu_model = NU_BRAUER
                mats[r].k1, mats[r].k2, mats[r].k3 = (float(v) for v in m.brauer)
                mats[r].bmax = float(m.bmax)
            else:
                mats[r].nu_model = NU_LINEAR
                mats[r].nu = float(m.nu)
        self._check(self._lib.pppc_set_mesh(
            self._h, xy.shape[0], xy.ctypes.data, tri.shape[0], tri.ctypes.data, region.ctypes.data,
            dirichlet.ctypes.data, len(materials), mats))
        self.n_nodes = xy.shape[0]

    def set_source(self, amp, freq, phase=None):
        amp = _as_host(np.atleast_1d(amp), np.float64)
        freq = _as_host(np.atleast_1d(freq), np.float64)
        phase = np.zeros_like(amp) if phase is None else _as_host(np.atleast_1d(phase), np.float64)
        self._check(self._lib.pppc_set_source(self._h, amp.size, amp.ctypes.data, freq.ctypes.data,
                                              phase.ctypes.data))

    @property
    def ndof(self) -> int:
        return int(self._lib.pppc_ndof(self._h))

    # -- state ---------------------------------------------------------------
    def _shape_ok(self, a):
        if tuple(a.shape) != (self.N, self.n_nodes):
            raise ValueError(f"state must have shape ({self.N}, {self.n_nodes}), got {tuple(a.shape)}")

    def _ptr_in(self, U):
        self._shape_ok(U)
        if _is_cuda_tensor(U):
            import torch
            if U.dtype != torch.float64 or not U.is_contiguous():
                raise ValueError("device states must be contiguous float64 tensors")
            return U, U.data_ptr(), 1
        a = _as_host(U, np.float64)
        return a, a.ctypes.data, 0

    def _out_like(self, like):
        if _is_cuda_tensor(like):
            import torch
            t = torch.empty((self.N, self.n_nodes), dtype=torch.float64, device=like.device)
            return t, t.data_ptr()
        a = np.empty((self.N, self.n_nodes))
        return a, a.ctypes.data

    def set_state(self, U):
        keep, ptr, dev = self._ptr_in(U)
        self._check(self._lib.pppc_set_state(self._h, ptr, dev))

    def get_state(self, device=None):
        if device is not None:
            import torch
            t = torch.empty((self.N, self.n_nodes), dtype=torch.float64, device=device)
            self._check(self._lib.pppc_get_state(self._h, t.data_ptr(), 1))
            return t
        a = np.empty((self.N, self.n_nodes))
        self._check(self._lib.pppc_get_state(self._h, a.ctypes.data, 0))
        return a

    # -- the method ------------------------------------------------------------
    def propagate_fine(self, U):
        """F[j] = F_{j+1}(U[j]) for all subintervals at once (Eqs. 2-3)."""
        keep, ptr, dev = self._ptr_in(U)
        out, optr = self._out_like(U)
        self._check(self._lib.pppc_propagate_fine(self._h, ptr, optr, dev))
        return out

    def propagate_fine_window(self, U, first: int, count: int):
        """Levels first..first+count of every subinterval: U[j] at T_j + first dt
        -> F[j] at T_j + (first + count) dt (Eq. 3 on part of each subinterval)."""
        keep, ptr, dev = self._ptr_in(U)
        out, optr = self._out_like(U)
        self._check(self._lib.pppc_propagate_fine_window(self._h, ptr, optr, int(first), int(count), dev))
        return out

    def coarse_update(self, U, F):
        """U^{k+1} from U^k and F^k (Eq. 4 through Eqs. 9-14); returns (U_new, rel_res)."""
        ku, pu, dev = self._ptr_in(U)
        kf, pf, devf = self._ptr_in(F)
        if dev != devf:
            raise ValueError("U and F must both be host or both be device arrays")
        out, optr = self._out_like(U)
        rr = ctypes.c_double()
        self._check(self._lib.pppc_coarse_update(self._h, pu, pf, optr, ctypes.byref(rr), dev))
        return out, rr.value

    def iterate(self) -> float:
        rr = ctypes.c_double()
        self._check(self._lib.pppc_iterate(self._h, ctypes.byref(rr)))
        return rr.value

    def solve_periodic(self, tol: float = 1e-8, kmax: int = 50, raise_on_fail: bool = True):
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        st = self._lib.pppc_solve_periodic(self._h, float(tol), int(kmax), ctypes.byref(it), ctypes.byref(rr))
        if st != 0 and (raise_on_fail or st != 9):
            self._check(st)
        return it.value, rr.value

    def set_trace(self, cap: int):
        """Record up to ``cap`` Newton records per fine sweep (0 turns it off)."""
        self._check(self._lib.pppc_set_trace(self._h, int(cap)))
        self._trace_cap = int(cap)

    def trace(self):
        """Records of the last fine sweep: rows of (step, Newton iteration,
        max ||R||, lanes iterating, PCG iterations before this test)."""
        cap = getattr(self, "_trace_cap", 0)
        out = np.zeros((max(cap, 1), 5))
        n = ctypes.c_int32()
        self._check(self._lib.pppc_get_trace(self._h, out.ctypes.data, cap, ctypes.byref(n)))
        return out[:min(n.value, cap)]

    def mesh_counts(self) -> dict:
        c = _lib.pppc_mesh_counts()
        self._check(self._lib.pppc_get_mesh_counts(self._h, ctypes.byref(c)))
        return {k: getattr(c, k) for k, _ in _lib.pppc_mesh_counts._fields_}

    def fine_plan(self) -> dict:
        """Lane-team split of the fine sweep in use and the tuner's timings."""
        p = _lib.pppc_fine_plan_info()
        self._check(self._lib.pppc_get_fine_plan(self._h, ctypes.byref(p)))
        n = p.n_candidates
        return {"lanes_per_team": p.lanes_per_team, "teams": p.teams, "threads_per_row": p.threads_per_row,
                "blocks_min": p.blocks_min, "blocks_max": p.blocks_max,
                "candidates": list(p.candidate_lanes[:n]), "candidate_ms": list(p.candidate_ms[:n]),
                "amg_rows": list(p.amg_rows[:p.amg_levels])}

    def stats(self) -> dict:
        s = pppc_stats()
        self._check(self._lib.pppc_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in pppc_stats._fields_}

    def adjoint(self, region: int, tol: float = 1e-10, kmax: int = 60):
        """Loss P [W/m] of the current (periodic) state and dP/d(sigma, k1, k2,
        k3) of region ``region`` by the periodic adjoint.  Returns
        (loss, grad[4], info)."""
        r = _lib.pppc_adjoint_result()
        self._check(self._lib.pppc_adjoint(self._h, int(region), float(tol), int(kmax), ctypes.byref(r)))
        info = {"iterations": r.iterations, "rel_res": r.rel_res, "forward_rel_res": r.forward_rel_res}
        return r.loss, np.array(list(r.grad)), info


def from_problem(problem, **cfg) -> PPPC:
    """Build a solver from any object shaped like ``synth.coax.Problem``
    (mesh arrays, per-region materials, excitation, time grid)."""
    mats = []
    for r in range(len(problem.sigma)):
        brauer = tuple(problem.brauer[r]) if int(problem.nu_model[r]) == NU_BRAUER else None
        bmax = float(problem.bmax[r]) if getattr(problem, "bmax", None) is not None else 0.0
        mats.append(Material(sigma=float(problem.sigma[r]), nu=float(problem.nu[r]), brauer=brauer,
                             is_source=bool(problem.is_source[r]), bmax=bmax))
    s = PPPC(problem.T, problem.N, problem.n_fine, **cfg)
    m = problem.mesh
    s.set_mesh(m.xy, m.tri, m.region, m.dirichlet, mats)
    s.set_source(problem.amp, problem.freq, problem.phase)
    return s


class PPPCBatch:
    """Many independent problems solved together (one team of blocks per
    member in each cooperative launch, two CUDA graphs per iteration).  The
    members are ``PPPC`` objects with mesh, source and state set; they keep
    their own states, so ``member.get_state()`` reads the result."""

    def __init__(self, members, autotune: bool = True):
        self._lib = _lib.load()
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        b = ctypes.c_void_p()
        _lib.check_batch(self._lib.pppc_batch_create(arr, len(self.members), int(bool(autotune)),
                                                     ctypes.byref(b)), None)
        self._b = b

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.pppc_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st):
        _lib.check_batch(st, self._b)

    def iterate(self) -> np.ndarray:
        rr = np.zeros(len(self.members))
        self._check(self._lib.pppc_batch_iterate(self._b, rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return rr

    def solve_periodic(self, tol: float = 1e-8, kmax: int = 50, raise_on_fail: bool = True):
        """Returns (iters[count], rel_res[count])."""
        its = np.zeros(len(self.members), dtype=np.int32)
        rr = np.zeros(len(self.members))
        st = self._lib.pppc_batch_solve_periodic(self._b, float(tol), int(kmax),
                                                 its.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                 rr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if raise_on_fail or st != 9:   # PPPC_ERR_NOT_CONVERGED
            self._check(st)
        return its, rr

    def teams(self):
        f = np.zeros(len(self.members), dtype=np.int32)
        c = np.zeros(len(self.members), dtype=np.int32)
        self._check(self._lib.pppc_batch_get_teams(self._b, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   c.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return f, c

    def lanes(self):
        """Per member: (lanes per team, teams) of its fine sweep in the batch."""
        lp = np.zeros(len(self.members), dtype=np.int32)
        tm = np.zeros(len(self.members), dtype=np.int32)
        self._check(self._lib.pppc_batch_get_lanes(self._b, lp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   tm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return lp, tm

    def stats(self) -> dict:
        s = _lib.pppc_batch_stats()
        self._check(self._lib.pppc_batch_get_stats(self._b, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.pppc_batch_stats._fields_}
