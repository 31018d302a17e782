"""Thin ctypes binding of the C ABI in include/amg.h (argument marshalling only).

Every computation runs in libamg.so's CUDA kernels. There is no CPU fallback:
if the library has not been built, ``lib()`` raises.

Device arrays are torch CUDA tensors (contiguous, int32 / float64); the
``*_host`` calls take numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libamg.so")

AMG_OK = 0
AMG_NOT_CONVERGED = 1
AMG_FP64 = 0
AMG_FP32_VCYCLE = 1
MAX_LEVELS = 32
MAX_SWEEPS = 8

STATUS_NAMES = {
    0: "AMG_OK", 1: "AMG_NOT_CONVERGED", -1: "AMG_ERR_ARG", -2: "AMG_ERR_NOT_SPD", -3: "AMG_ERR_BAD_W",
    -4: "AMG_ERR_OOM", -5: "AMG_ERR_CUDA", -6: "AMG_ERR_BREAKDOWN", -7: "AMG_ERR_TIMEOUT",
    -8: "AMG_ERR_TOO_LARGE", -9: "AMG_ERR_BUDGET",
}
globals().update({name: code for code, name in STATUS_NAMES.items()})

EXPORTED = [
    "amg_options_default", "amg_setup", "amg_setup_host", "amg_solve", "amg_solve_host", "amg_vcycle",
    "amg_hierarchy_info", "amg_export_level", "amg_sweep_dims", "amg_export_sweep", "amg_coarse_factor",
    "amg_free", "amg_last_error", "amg_kernel_stats_count", "amg_kernel_stats", "amg_kernel_stats_reset",
    "amg_launch_count", "amg_match_noalloc", "amg_solve_batch", "amg_serve_create", "amg_serve_submit",
    "amg_serve_step", "amg_serve_poll", "amg_serve_stats_get", "amg_serve_free", "amg_setup_many",
    "amg_solve_many", "amg_system_offsets", "amg_tune_save", "amg_tune_load", "amg_tune_clear", "amg_tune_size",
    "amg_smooth_vector", "amg_pbar_nnz", "amg_export_pbar",
]
KCYCLE_FULL = 32
NOALLOC_MAX_N = 65536
NOALLOC_MAX_NNZ = 524288


class amg_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int32), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class amg_options(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("max_coarse", ctypes.c_int), ("max_levels", ctypes.c_int),
                ("pre", ctypes.c_int), ("post", ctypes.c_int), ("omega", ctypes.c_double),
                ("precision", ctypes.c_int), ("max_dense", ctypes.c_int), ("keep_sweeps", ctypes.c_int),
                ("profile", ctypes.c_int), ("match_kernel", ctypes.c_int), ("krylov", ctypes.c_int),
                ("cycle", ctypes.c_int), ("smooth_p", ctypes.c_int), ("autotune", ctypes.c_int),
                ("omega_rule", ctypes.c_int), ("min_ratio", ctypes.c_double), ("stream", ctypes.c_void_p)]


class amg_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("relres", ctypes.c_double),
                ("true_relres", ctypes.c_double), ("solve_ms", ctypes.c_double)]


class amg_hier_info(ctypes.Structure):
    _fields_ = [("num_levels", ctypes.c_int), ("n", ctypes.c_int64 * MAX_LEVELS),
                ("nnz", ctypes.c_int64 * MAX_LEVELS), ("sweeps_done", ctypes.c_int * MAX_LEVELS),
                ("rounds", (ctypes.c_int * MAX_SWEEPS) * MAX_LEVELS), ("opc", ctypes.c_double),
                ("avg_coarsening_ratio", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("coarse_solver", ctypes.c_int), ("device_bytes", ctypes.c_size_t)]


class amg_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("columns_completed", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("columns_per_s", ctypes.c_double), ("elapsed_s", ctypes.c_double),
                ("budget_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t)]


class AmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib() -> ctypes.CDLL:
    """Load libamg.so; raise if it is missing (build it with build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        L.amg_options_default.argtypes = [ctypes.POINTER(amg_options)]
        L.amg_options_default.restype = None
        for name in ("amg_setup", "amg_setup_host"):
            f = getattr(L, name)
            f.argtypes = [ctypes.POINTER(amg_csr), _vp, ctypes.POINTER(amg_options), ctypes.POINTER(_vp)]
            f.restype = ctypes.c_int
        for name in ("amg_solve", "amg_solve_host"):
            f = getattr(L, name)
            f.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(amg_solve_info)]
            f.restype = ctypes.c_int
        L.amg_solve_batch.argtypes = [_vp, ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(amg_solve_info)]
        L.amg_solve_batch.restype = ctypes.c_int
        L.amg_serve_create.argtypes = [ctypes.c_int, ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t,
                                       ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp)]
        L.amg_serve_create.restype = ctypes.c_int
        L.amg_serve_submit.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _i64p]
        L.amg_serve_submit.restype = ctypes.c_int
        L.amg_serve_step.argtypes = [_vp, _i64p]
        L.amg_serve_step.restype = ctypes.c_int
        L.amg_serve_poll.argtypes = [_vp, _i64p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.c_int]
        L.amg_serve_poll.restype = ctypes.c_int
        L.amg_serve_stats_get.argtypes = [_vp, ctypes.POINTER(amg_serve_stats)]
        L.amg_serve_stats_get.restype = ctypes.c_int
        L.amg_serve_free.argtypes = [_vp]
        L.amg_serve_free.restype = None
        L.amg_setup_many.argtypes = [ctypes.c_int, ctypes.POINTER(amg_csr), ctypes.POINTER(_vp),
                                     ctypes.POINTER(amg_options), ctypes.POINTER(_vp)]
        L.amg_setup_many.restype = ctypes.c_int
        L.amg_solve_many.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(amg_solve_info)]
        L.amg_solve_many.restype = ctypes.c_int
        L.amg_system_offsets.argtypes = [_vp, _i32p]
        L.amg_system_offsets.restype = ctypes.c_int
        L.amg_vcycle.argtypes = [_vp, _vp, _vp]
        L.amg_vcycle.restype = ctypes.c_int
        L.amg_hierarchy_info.argtypes = [_vp, ctypes.POINTER(amg_hier_info)]
        L.amg_hierarchy_info.restype = ctypes.c_int
        L.amg_export_level.argtypes = [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.amg_export_level.restype = ctypes.c_int
        L.amg_sweep_dims.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _i64p]
        L.amg_sweep_dims.restype = ctypes.c_int
        L.amg_export_sweep.argtypes = [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.amg_export_sweep.restype = ctypes.c_int
        L.amg_coarse_factor.argtypes = [_vp, _vp]
        L.amg_coarse_factor.restype = ctypes.c_int
        L.amg_free.argtypes = [_vp]
        L.amg_free.restype = None
        L.amg_last_error.argtypes = []
        L.amg_last_error.restype = ctypes.c_char_p
        L.amg_kernel_stats_count.argtypes = []
        L.amg_kernel_stats_count.restype = ctypes.c_int
        L.amg_kernel_stats.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), _i64p,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.amg_kernel_stats.restype = ctypes.c_int
        L.amg_kernel_stats_reset.argtypes = [_vp]
        L.amg_kernel_stats_reset.restype = ctypes.c_int
        L.amg_match_noalloc.argtypes = [ctypes.POINTER(amg_csr), _vp, _vp, _vp, _i32p]
        L.amg_match_noalloc.restype = ctypes.c_int
        L.amg_launch_count.argtypes = []
        L.amg_launch_count.restype = ctypes.c_int64
        for name in ("amg_tune_save", "amg_tune_load"):
            getattr(L, name).argtypes = [ctypes.c_char_p]
            getattr(L, name).restype = ctypes.c_int
        L.amg_pbar_nnz.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
        L.amg_pbar_nnz.restype = ctypes.c_int
        L.amg_export_pbar.argtypes = [_vp, ctypes.c_int, _i32p, _i32p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.amg_export_pbar.restype = ctypes.c_int
        L.amg_smooth_vector.argtypes = [ctypes.POINTER(amg_csr), _vp, _vp, ctypes.c_int, ctypes.c_double, _vp]
        L.amg_smooth_vector.restype = ctypes.c_int
        L.amg_tune_clear.argtypes = []
        L.amg_tune_clear.restype = None
        L.amg_tune_size.argtypes = []
        L.amg_tune_size.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status):
    if status < 0:
        raise AmgError(status, lib().amg_last_error().decode())
    return status


def amg_options_default(**overrides) -> amg_options:
    o = amg_options()
    lib().amg_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream":
            v = ctypes.c_void_p(v)
        setattr(o, k, v)
    return o


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Hierarchy:
    """Owns an amg_hierarchy*; freed by close() or garbage collection."""

    def __init__(self, handle, n):
        self._h = handle
        self.n = n

    @property
    def handle(self):
        if not self._h:
            raise ValueError("hierarchy was freed")
        return self._h

    def close(self):
        if self._h:
            lib().amg_free(self._h)
            self._h = None

    __del__ = close


def amg_setup(row_ptr, col, val, w, host: bool = False, **opts) -> Hierarchy:
    """Builds the hierarchy from a CSR matrix and smooth vector w.

    Device tensors (torch, cuda) unless host=True (numpy). Options as in amg_options.
    """
    n = int(row_ptr.shape[0] - 1)
    A = amg_csr(n, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val))
    if "stream" not in opts and not host:
        opts["stream"] = _current_stream()
    o = amg_options_default(**opts)
    h = ctypes.c_void_p()
    f = lib().amg_setup_host if host else lib().amg_setup
    _check(f(ctypes.byref(A), _ptr(w), ctypes.byref(o), ctypes.byref(h)))
    return Hierarchy(h.value, n)


def amg_setup_host(row_ptr, col, val, w, **opts) -> Hierarchy:
    return amg_setup(row_ptr, col, val, w, host=True, **opts)


def _info_dict(inf, status):
    return dict(status=status, iterations=inf.iterations, restarts=inf.restarts, relres=inf.relres,
                true_relres=inf.true_relres, solve_ms=inf.solve_ms)


def amg_solve(h: Hierarchy, b, x, rtol: float = 1e-6, maxit: int = 1000) -> dict:
    """PCG with the V-cycle preconditioner; x holds x0 on entry (device tensors)."""
    inf = amg_solve_info()
    st = _check(lib().amg_solve(h.handle, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(inf)))
    return _info_dict(inf, st)


def amg_solve_host(h: Hierarchy, b: np.ndarray, x: np.ndarray, rtol: float = 1e-6, maxit: int = 1000) -> dict:
    inf = amg_solve_info()
    st = _check(lib().amg_solve_host(h.handle, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(inf)))
    return _info_dict(inf, st)


def amg_solve_batch(h: Hierarchy, B, X, rtol: float = 1e-6, maxit: int = 1000) -> list:
    """Block solve of row-major n x k device tensors B (read) and X (x0 in, solution out)."""
    k = int(B.shape[1])
    infos = (amg_solve_info * k)()
    st = _check(lib().amg_solve_batch(h.handle, k, _ptr(B), _ptr(X), float(rtol), int(maxit), infos))
    return [dict(_info_dict(infos[c], st)) for c in range(k)]


def amg_setup_many(systems, **opts) -> Hierarchy:
    """One hierarchy for the block-diagonal union of systems [(row_ptr, col, val, w), ...] (device tensors)."""
    m = len(systems)
    arr = (amg_csr * m)()
    ws = (ctypes.c_void_p * m)()
    for i, (rp, cl, vl, w) in enumerate(systems):
        arr[i] = amg_csr(int(rp.shape[0] - 1), int(cl.shape[0]), _ptr(rp), _ptr(cl), _ptr(vl))
        ws[i] = _ptr(w)
    if "stream" not in opts:
        opts["stream"] = _current_stream()
    o = amg_options_default(**opts)
    h = ctypes.c_void_p()
    _check(lib().amg_setup_many(m, arr, ws, ctypes.byref(o), ctypes.byref(h)))
    n = sum(int(rp.shape[0] - 1) for rp, _, _, _ in systems)
    return Hierarchy(h.value, n)


def amg_solve_many(h: Hierarchy, b, x, m: int, rtol: float = 1e-6, maxit: int = 1000) -> list:
    """One CG per system on concatenated device vectors b, x; returns m info dicts."""
    infos = (amg_solve_info * m)()
    st = _check(lib().amg_solve_many(h.handle, _ptr(b), _ptr(x), float(rtol), int(maxit), infos))
    return [_info_dict(infos[s], st) for s in range(m)]


def amg_system_offsets(h: Hierarchy, m: int) -> np.ndarray:
    off = np.empty(m + 1, dtype=np.int32)
    _check(lib().amg_system_offsets(h.handle, off.ctypes.data_as(_i32p)))
    return off


def amg_vcycle(h: Hierarchy, r, z) -> None:
    _check(lib().amg_vcycle(h.handle, _ptr(r), _ptr(z)))


def amg_hierarchy_info(h: Hierarchy) -> dict:
    inf = amg_hier_info()
    _check(lib().amg_hierarchy_info(h.handle, ctypes.byref(inf)))
    nl = inf.num_levels
    return dict(num_levels=nl, n=[inf.n[i] for i in range(nl)], nnz=[inf.nnz[i] for i in range(nl)],
                sweeps_done=[inf.sweeps_done[i] for i in range(nl)],
                rounds=[[inf.rounds[i][s] for s in range(inf.sweeps_done[i])] for i in range(nl)],
                opc=inf.opc, avg_coarsening_ratio=inf.avg_coarsening_ratio, setup_ms=inf.setup_ms,
                coarse_solver=inf.coarse_solver, device_bytes=inf.device_bytes)


def amg_export_level(h: Hierarchy, level: int) -> dict:
    info = amg_hierarchy_info(h)
    n, nnz = info["n"][level], info["nnz"][level]
    last = level == info["num_levels"] - 1
    out = dict(n=n, nnz=nnz, row_ptr=np.empty(n + 1, np.int32), col=np.empty(nnz, np.int32),
               val=np.empty(nnz), w=np.empty(n), minv=np.empty(n),
               agg=None if last else np.empty(n, np.int32), p=None if last else np.empty(n))
    _check(lib().amg_export_level(h.handle, level, _ptr(out["row_ptr"]), _ptr(out["col"]), _ptr(out["val"]),
                                  _ptr(out["w"]), _ptr(out["minv"]), _ptr(out["agg"]), _ptr(out["p"])))
    return out


def amg_export_sweep(h: Hierarchy, level: int, sweep: int) -> dict:
    n, nc, nnzc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().amg_sweep_dims(h.handle, level, sweep, ctypes.byref(n), ctypes.byref(nc), ctypes.byref(nnzc)))
    out = dict(n=n.value, nc=nc.value, nnz_c=nnzc.value, mate=np.empty(n.value, np.int32),
               agg=np.empty(n.value, np.int32), p=np.empty(n.value), wc=np.empty(nc.value))
    _check(lib().amg_export_sweep(h.handle, level, sweep, _ptr(out["mate"]), _ptr(out["agg"]), _ptr(out["p"]),
                                  _ptr(out["wc"])))
    return out


def amg_coarse_factor(h: Hierarchy) -> np.ndarray:
    info = amg_hierarchy_info(h)
    nc = info["n"][-1]
    L = np.empty(nc * nc)
    _check(lib().amg_coarse_factor(h.handle, _ptr(L)))
    return L.reshape(nc, nc).T.copy()


def amg_free(h: Hierarchy) -> None:
    h.close()


def amg_kernel_stats(h: Hierarchy) -> dict:
    """{name: (timed scopes, total ms, algorithmic bytes)} for scopes that ran (needs profile=1)."""
    out = {}
    for idx in range(lib().amg_kernel_stats_count()):
        name = ctypes.c_char_p()
        sc = ctypes.c_int64()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        _check(lib().amg_kernel_stats(h.handle, idx, ctypes.byref(name), ctypes.byref(sc), ctypes.byref(ms),
                                      ctypes.byref(by)))
        if sc.value:
            out[name.value.decode()] = (sc.value, ms.value, by.value)
    return out


def amg_kernel_stats_reset(h: Hierarchy) -> None:
    _check(lib().amg_kernel_stats_reset(h.handle))


def amg_export_pbar(h: Hierarchy, level: int) -> dict:
    """Smoothed prolongator of a level (hierarchies built with smooth_p=1) as host arrays."""
    nnz = ctypes.c_int64()
    _check(lib().amg_pbar_nnz(h.handle, level, ctypes.byref(nnz)))
    n = amg_hierarchy_info(h)["n"][level]
    rp = np.empty(n + 1, dtype=np.int32)
    cl = np.empty(nnz.value, dtype=np.int32)
    vl = np.empty(nnz.value, dtype=np.float64)
    om = ctypes.c_double()
    _check(lib().amg_export_pbar(h.handle, level, rp.ctypes.data_as(_i32p), cl.ctypes.data_as(_i32p),
                                 vl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(om)))
    return dict(row_ptr=rp, col=cl, val=vl, omega=om.value)


def amg_smooth_vector(row_ptr, col, val, w0, sweeps: int, omega: float = 1.0, stream=None):
    """Smooth vector for amg_setup: `sweeps` l1-Jacobi iterations on A w = 0 from w0 (device tensors)."""
    import torch
    A = amg_csr(int(row_ptr.shape[0] - 1), int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val))
    w = torch.empty_like(w0)
    st = stream if stream is not None else _current_stream()
    _check(lib().amg_smooth_vector(ctypes.byref(A), _ptr(w0), _ptr(w), int(sweeps), float(omega), st))
    return w


def amg_tune_save(path: str) -> None:
    """Write the launch-shape cache of the autotuner to a text file."""
    _check(lib().amg_tune_save(os.fsencode(path)))


def amg_tune_load(path: str) -> None:
    """Merge a launch-shape cache file into the process cache."""
    _check(lib().amg_tune_load(os.fsencode(path)))


def amg_tune_clear() -> None:
    lib().amg_tune_clear()


def amg_tune_size() -> int:
    return int(lib().amg_tune_size())


def amg_launch_count() -> int:
    return int(lib().amg_launch_count())


def amg_match_noalloc(row_ptr, col, val, w, mate, stream=None) -> int:
    """Matching of (A, w) into the device tensor `mate` without any device allocation.

    For callers that may not allocate when they need it (all device memory
    reserved at start-up for their own pool or budget, or no allocation allowed
    after start-up). Uses the library's fixed scratch array, so
    n <= NOALLOC_MAX_N and nnz <= NOALLOC_MAX_NNZ; calls must not overlap on
    the GPU. Returns the number of matching rounds.
    """
    n = int(row_ptr.shape[0] - 1)
    A = amg_csr(n, int(col.shape[0]), _ptr(row_ptr), _ptr(col), _ptr(val))
    rounds = ctypes.c_int32(0)
    st = _current_stream() if stream is None else stream
    _check(lib().amg_match_noalloc(ctypes.byref(A), _ptr(w), _ptr(mate), ctypes.c_void_p(st), ctypes.byref(rounds)))
    return rounds.value


class Server:
    """Continuous-batching solve server over cached hierarchies (amg_serve_*).

    Host numpy arrays are kept referenced until their request completes.
    """

    def __init__(self, hierarchies, slots=16, budget_bytes=1 << 40, rtol=1e-6, maxit=1000):
        arr = (ctypes.c_void_p * len(hierarchies))(*[h.handle for h in hierarchies])
        out = ctypes.c_void_p()
        _check(lib().amg_serve_create(len(hierarchies), arr, int(slots), int(budget_bytes), float(rtol), int(maxit),
                                      ctypes.byref(out)))
        self._s = out.value
        self._hier = list(hierarchies)
        self._live = {}

    def submit(self, hid, B):
        """Queue the columns of host array B (n x k); returns (id, X) with X filled at completion."""
        B = np.ascontiguousarray(B if B.ndim == 2 else B[:, None], dtype=np.float64)
        X = np.zeros_like(B)
        rid = ctypes.c_int64()
        _check(lib().amg_serve_submit(self._s, int(hid), int(B.shape[1]), _ptr(B), _ptr(X), ctypes.byref(rid)))
        self._live[rid.value] = (B, X)
        return rid.value, X

    def step(self) -> int:
        pending = ctypes.c_int64()
        _check(lib().amg_serve_step(self._s, ctypes.byref(pending)))
        return pending.value

    def poll(self, max_items=256):
        ids = (ctypes.c_int64 * max_items)()
        st = (ctypes.c_int * max_items)()
        lat = (ctypes.c_double * max_items)()
        it = (ctypes.c_int * max_items)()
        rel = (ctypes.c_double * max_items)()
        n = lib().amg_serve_poll(self._s, ids, st, lat, it, rel, max_items)
        out = []
        for i in range(n):
            B, X = self._live.pop(ids[i])
            out.append(dict(id=ids[i], status=st[i], latency_ms=lat[i], iterations=it[i], relres=rel[i], X=X))
        return out

    def stats(self) -> dict:
        s = amg_serve_stats()
        _check(lib().amg_serve_stats_get(self._s, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in amg_serve_stats._fields_}

    def close(self):
        if getattr(self, "_s", None):
            lib().amg_serve_free(self._s)
            self._s = None

    __del__ = close
