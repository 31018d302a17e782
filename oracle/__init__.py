"""Python loader for the FP64 CPU oracle (amg_oracle.cpp).

TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package. The CUDA library never uses it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction) into liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_setup.restype = ctypes.c_void_p
            L.orc_setup.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, _ip]
            L.orc_coarse_is_cg.argtypes = [ctypes.c_void_p]
            L.orc_set_cycle.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_smooth_vector.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, ctypes.c_int, ctypes.c_double,
                                            _f64p]
            L.orc_setup_seg.restype = ctypes.c_void_p
            L.orc_setup_seg.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, _i32p, ctypes.c_int, ctypes.c_int,
                                        _ip]
            L.orc_level_pbar_nnz.restype = ctypes.c_int64
            L.orc_level_pbar_nnz.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_level_pbar.restype = ctypes.c_double
            L.orc_level_pbar.argtypes = [ctypes.c_void_p, ctypes.c_int, _i32p, _i32p, _f64p]
            for name in ("orc_free",):
                getattr(L, name).argtypes = [ctypes.c_void_p]
            L.orc_num_levels.argtypes = [ctypes.c_void_p]
            L.orc_level_dims.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip, _i64p]
            L.orc_level_csr.argtypes = [ctypes.c_void_p, ctypes.c_int, _i32p, _i32p, _f64p]
            L.orc_level_vectors.argtypes = [ctypes.c_void_p, ctypes.c_int, _f64p, _f64p]
            L.orc_level_prolongator.argtypes = [ctypes.c_void_p, ctypes.c_int, _i32p, _f64p]
            L.orc_level_num_sweeps.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.orc_sweep_dims.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _ip, _ip, _i64p, _ip]
            L.orc_sweep_data.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _f64p, _f64p]
            L.orc_coarse_factor.argtypes = [ctypes.c_void_p, _f64p]
            L.orc_vcycle.argtypes = [ctypes.c_void_p, _f64p, _f64p]
            L.orc_vcycle_level.argtypes = [ctypes.c_void_p, ctypes.c_int, _f64p, _f64p]
            L.orc_pcg.argtypes = [ctypes.c_void_p, _f64p, _f64p, ctypes.c_double, ctypes.c_int, ctypes.c_int, _ip,
                                  _f64p, _f64p]
            L.orc_weights.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _f64p]
            L.orc_match_greedy.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _i32p]
            L.orc_match_ld.argtypes = [ctypes.c_int, _i32p, _i32p, _f64p, _f64p, _i32p, _ip]
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr_args(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = np.ascontiguousarray(A.val, dtype=np.float64)
    return rp, cl, vl


class OracleError(RuntimeError):
    pass


def weights(A, w):
    rp, cl, vl = _csr_args(A)
    w = np.ascontiguousarray(w, dtype=np.float64)
    c = np.empty(A.nnz)
    e = lib().orc_weights(A.n, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p), _p(w, _f64p), _p(c, _f64p))
    if e:
        raise OracleError(f"orc_weights: {e}")
    return c


def match_greedy(A, w):
    rp, cl, vl = _csr_args(A)
    w = np.ascontiguousarray(w, dtype=np.float64)
    m = np.empty(A.n, dtype=np.int32)
    e = lib().orc_match_greedy(A.n, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p), _p(w, _f64p), _p(m, _i32p))
    if e:
        raise OracleError(f"orc_match_greedy: {e}")
    return m


def match_ld(A, w):
    rp, cl, vl = _csr_args(A)
    w = np.ascontiguousarray(w, dtype=np.float64)
    m = np.empty(A.n, dtype=np.int32)
    r = ctypes.c_int(0)
    e = lib().orc_match_ld(A.n, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p), _p(w, _f64p), _p(m, _i32p),
                           ctypes.byref(r))
    if e:
        raise OracleError(f"orc_match_ld: {e}")
    return m, r.value


def smooth_vector(A, w0, sweeps, omega=1.0):
    """`sweeps` l1-Jacobi iterations on A w = 0 from w0 (Section 3.2)."""
    rp, cl, vl = _csr_args(A)
    w0 = np.ascontiguousarray(w0, dtype=np.float64)
    w = np.empty(A.n)
    lib().orc_smooth_vector(A.n, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p), _p(w0, _f64p), int(sweeps),
                            float(omega), _p(w, _f64p))
    return w


class Level:
    __slots__ = ("n", "nnz", "row_ptr", "col", "val", "w", "minv", "agg", "p", "sweeps")


class Hierarchy:
    """Oracle hierarchy: setup in the constructor, then V-cycle and PCG."""

    def __init__(self, A, w=None, sweeps=3, max_coarse=200, max_levels=32, pre=1, post=1, omega=1.0,
                 use_ld=False, min_ratio=1.5, max_dense=4096, seg=None, cycle=0, smooth_p=False, omega_rule=0):
        rp, cl, vl = _csr_args(A)
        w = np.ones(A.n) if w is None else np.ascontiguousarray(w, dtype=np.float64)
        st = ctypes.c_int(0)
        sg = np.ascontiguousarray(seg if seg is not None else [0], dtype=np.int32)
        self._h = lib().orc_setup_seg(A.n, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p), _p(w, _f64p), sweeps,
                                      max_coarse, max_levels, pre, post, float(omega), int(use_ld), float(min_ratio),
                                      int(max_dense), 0 if seg is None else len(sg) - 1, _p(sg, _i32p),
                                      int(smooth_p), int(omega_rule), ctypes.byref(st))
        if not self._h:
            raise OracleError(f"orc_setup failed: {st.value}")
        lib().orc_set_cycle(self._h, int(cycle))
        self.n = A.n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return lib().orc_num_levels(self._h)

    def level(self, l: int) -> Level:
        L = lib()
        n = ctypes.c_int(0)
        nnz = ctypes.c_int64(0)
        L.orc_level_dims(self._h, l, ctypes.byref(n), ctypes.byref(nnz))
        lv = Level()
        lv.n, lv.nnz = n.value, nnz.value
        lv.row_ptr = np.empty(lv.n + 1, dtype=np.int32)
        lv.col = np.empty(lv.nnz, dtype=np.int32)
        lv.val = np.empty(lv.nnz)
        L.orc_level_csr(self._h, l, _p(lv.row_ptr, _i32p), _p(lv.col, _i32p), _p(lv.val, _f64p))
        lv.w = np.empty(lv.n)
        lv.minv = np.empty(lv.n)
        L.orc_level_vectors(self._h, l, _p(lv.w, _f64p), _p(lv.minv, _f64p))
        lv.agg = lv.p = None
        if l < self.num_levels - 1:
            lv.agg = np.empty(lv.n, dtype=np.int32)
            lv.p = np.empty(lv.n)
            L.orc_level_prolongator(self._h, l, _p(lv.agg, _i32p), _p(lv.p, _f64p))
        lv.sweeps = []
        for s in range(L.orc_level_num_sweeps(self._h, l)):
            ns, nc, nnzc, rounds = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_int(0)
            L.orc_sweep_dims(self._h, l, s, ctypes.byref(ns), ctypes.byref(nc), ctypes.byref(nnzc),
                             ctypes.byref(rounds))
            mate = np.empty(ns.value, dtype=np.int32)
            agg = np.empty(ns.value, dtype=np.int32)
            p = np.empty(ns.value)
            wc = np.empty(nc.value)
            L.orc_sweep_data(self._h, l, s, _p(mate, _i32p), _p(agg, _i32p), _p(p, _f64p), _p(wc, _f64p))
            lv.sweeps.append(dict(n=ns.value, nc=nc.value, nnz_c=nnzc.value, rounds=rounds.value, mate=mate,
                                  agg=agg, p=p, wc=wc))
        return lv

    def pbar(self, l: int):
        """Smoothed prolongator of level l as (Csr, omega) (hierarchies built with smooth_p)."""
        from paper_2006_16147_gb300.workloads import Csr
        n = self.sizes()[l][0]
        nnz = lib().orc_level_pbar_nnz(self._h, l)
        rp = np.empty(n + 1, dtype=np.int32)
        cl = np.empty(nnz, dtype=np.int32)
        vl = np.empty(nnz)
        om = lib().orc_level_pbar(self._h, l, _p(rp, _i32p), _p(cl, _i32p), _p(vl, _f64p))
        return Csr(rp, cl, vl), om

    def level_csr(self, l: int):
        from paper_2006_16147_gb300.workloads import Csr
        lv = self.level(l)
        return Csr(lv.row_ptr, lv.col, lv.val)

    def sizes(self):
        out = []
        for l in range(self.num_levels):
            n = ctypes.c_int(0)
            nnz = ctypes.c_int64(0)
            lib().orc_level_dims(self._h, l, ctypes.byref(n), ctypes.byref(nnz))
            out.append((n.value, nnz.value))
        return out

    @property
    def coarse_is_cg(self) -> bool:
        return bool(lib().orc_coarse_is_cg(self._h))

    def coarse_factor(self) -> np.ndarray:
        nc = self.sizes()[-1][0]
        L = np.empty(nc * nc)
        lib().orc_coarse_factor(self._h, _p(L, _f64p))
        return L.reshape(nc, nc).T.copy()   # column-major -> dense lower-triangular

    def vcycle(self, r, level: int = 0) -> np.ndarray:
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty_like(r)
        lib().orc_vcycle_level(self._h, level, _p(r, _f64p), _p(z, _f64p))
        return z

    def pcg(self, b, x0=None, rtol=1e-6, maxit=1000, flexible=False):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        tr = ctypes.c_double(0)
        st = lib().orc_pcg(self._h, _p(b, _f64p), _p(x, _f64p), float(rtol), int(maxit), int(flexible), ctypes.byref(it),
                           ctypes.byref(rr), ctypes.byref(tr))
        return x, dict(status=st, iterations=it.value, relres=rr.value, true_relres=tr.value)
