"""ctypes front end of the FP64 CPU oracle — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
import build as _build  # noqa: E402

_lib = None

_dp = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)
_u8 = C.POINTER(C.c_uint8)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_value.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_value.restype = C.c_int
        L.orc_walsh_subset.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint32]
        L.orc_walsh_subset.restype = C.c_double
        L.orc_walsh_by_size.argtypes = [C.c_int, C.c_int, C.c_int, _dp]
        L.orc_walsh_by_size.restype = None
        for name in ("orc_fe_walsh_bruteforce", "orc_fe_corners", "orc_fe_esp", "orc_fe_paper", "orc_fe_dp", "orc_fe"):
            fn = getattr(L, name)
            fn.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
            fn.restype = C.c_double
        L.orc_fe_or.argtypes = [C.c_int, _dp, _dp]
        L.orc_fe_or.restype = C.c_double
        L.orc_fe_xor.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.orc_fe_xor.restype = C.c_double
        L.orc_esp.argtypes = [C.c_int, _dp, _dp]
        L.orc_esp.restype = None
        L.orc_paper_ftilde.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp]
        L.orc_paper_ftilde.restype = None
        L.orc_eval_grad.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, _dp, C.c_int32, _dp, _dp, _dp, C.c_int, C.c_int]
        L.orc_eval_grad.restype = C.c_int
        L.orc_eval_scale.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, _dp, C.c_int32, _dp, _dp, _dp,
                                     C.c_double, C.c_int, C.c_int]
        L.orc_eval_scale.restype = C.c_int
        L.orc_check.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, C.c_int32, _dp, _u8, _i32, C.c_int]
        L.orc_check.restype = C.c_int
        L.orc_unsat_counts.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, C.c_int32, _dp, _i32]
        L.orc_unsat_counts.restype = C.c_int
        L.orc_erwa.argtypes = [C.c_int32, _i32, C.c_double, _dp]
        L.orc_erwa.restype = None
        L.orc_step_pgfp.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, _dp, C.c_int32, _dp, C.c_int32,
                                    C.c_double, C.c_double, C.c_int32, C.c_double, C.c_double, C.c_uint64,
                                    C.c_uint64, C.c_uint64, C.c_int, _u8, _i32, _i32, _dp, C.c_int]
        L.orc_step_pgfp.restype = C.c_int
        L.orc_rephase.argtypes = [C.c_int32, C.c_int32, _dp, C.c_int, _u8, C.c_uint64, C.c_uint64, C.c_uint64]
        L.orc_rephase.restype = C.c_int
        L.orc_splitmix64.argtypes = [C.c_uint64]
        L.orc_splitmix64.restype = C.c_uint64
        L.orc_uniform.argtypes = [C.c_uint64] * 4
        L.orc_uniform.restype = C.c_double
        L.orc_step.argtypes = [C.c_int32, C.c_int32, _i64, _i32, _u8, _i32, _dp, C.c_int32, _dp, C.c_int32, C.c_double,
                               C.c_uint64, C.c_uint64, C.c_uint64, C.c_int, _u8, _i32, C.c_int]
        L.orc_step.restype = C.c_int
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------------------------
# Per-constraint routines
# ---------------------------------------------------------------------------------------------

OR, XOR, ATLEAST = 0, 1, 2
_ROUTES = {"bruteforce": "orc_fe_walsh_bruteforce", "corners": "orc_fe_corners", "esp": "orc_fe_esp",
           "paper": "orc_fe_paper", "dp": "orc_fe_dp", "default": "orc_fe"}


def value(ctype: int, param: int, L: int, s: int) -> int:
    return lib().orc_value(ctype, param, L, s)


def walsh_subset(ctype, param, L, mask) -> float:
    return lib().orc_walsh_subset(ctype, param, L, mask)


def walsh_by_size(ctype, param, L) -> np.ndarray:
    a = np.zeros(L + 1)
    lib().orc_walsh_by_size(ctype, param, L, _p(a, _dp))
    return a


def esp(y) -> np.ndarray:
    y = _f64(y)
    e = np.zeros(len(y) + 1)
    lib().orc_esp(len(y), _p(y, _dp), _p(e, _dp))
    return e


def fe(ctype, param, y, route="default"):
    """(FE, dFE/dy) of one constraint at literal values y."""
    y = _f64(y)
    dy = np.zeros(max(len(y), 1))
    v = getattr(lib(), _ROUTES[route])(ctype, param, len(y), _p(y, _dp), _p(dy, _dp))
    return v, dy[: len(y)]


def fe_or(y):
    y = _f64(y)
    dy = np.zeros(max(len(y), 1))
    v = lib().orc_fe_or(len(y), _p(y, _dp), _p(dy, _dp))
    return v, dy[: len(y)]


def fe_xor(param, y):
    y = _f64(y)
    dy = np.zeros(max(len(y), 1))
    v = lib().orc_fe_xor(param, len(y), _p(y, _dp), _p(dy, _dp))
    return v, dy[: len(y)]


def paper_ftilde(ctype, param, L) -> np.ndarray:
    re = np.zeros(L + 1)
    im = np.zeros(L + 1)
    lib().orc_paper_ftilde(ctype, param, L, _p(re, _dp), _p(im, _dp))
    return re + 1j * im


# ---------------------------------------------------------------------------------------------
# Instance-level routines
# ---------------------------------------------------------------------------------------------

_ROUTE_ID = {"default": 0, "dp": 1, "esp": 2, "paper": 3}


def _inst_arrays(inst):
    return (np.ascontiguousarray(inst.row_ptr, dtype=np.int64), np.ascontiguousarray(inst.lits, dtype=np.int32),
            np.ascontiguousarray(inst.ctype, dtype=np.uint8), np.ascontiguousarray(inst.param, dtype=np.int32),
            np.ascontiguousarray(inst.weights, dtype=np.float64))


def eval_grad(inst, x, nthreads: int = 0, route: str = "default", weights=None):
    """F(x_b) and grad F(x_b) for x [B, n] (any float dtype, converted exactly to float64)."""
    rp, lits, ty, pa, w = _inst_arrays(inst)
    if weights is not None:
        w = _f64(weights)
    x = _f64(np.atleast_2d(x))
    B = x.shape[0]
    f = np.zeros(B)
    g = np.zeros_like(x)
    rc = lib().orc_eval_grad(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), _p(w, _dp),
                             B, _p(x, _dp), _p(f, _dp), _p(g, _dp), nthreads, _ROUTE_ID[route])
    if rc != 0:
        raise ValueError("oracle: bad input (variable out of range or NaN)")
    return f, g


def eval_scale(inst, x, floor: float = 0.0, nthreads: int = 0, weights=None, floor_types=(ATLEAST,)):
    """Condition scales (sum_c w|FE_c|, A[b,v] = sum_{c ni v} w max(|dFE_c/dy_v|, floor)) at x;
    the floor applies to constraints whose type is in floor_types."""
    rp, lits, ty, pa, w = _inst_arrays(inst)
    if weights is not None:
        w = _f64(weights)
    x = _f64(np.atleast_2d(x))
    B = x.shape[0]
    sf = np.zeros(B)
    A = np.zeros_like(x)
    rc = lib().orc_eval_scale(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), _p(w, _dp),
                              B, _p(x, _dp), _p(sf, _dp), _p(A, _dp), float(floor),
                              sum(1 << t for t in floor_types), nthreads)
    if rc != 0:
        raise ValueError("oracle: bad input")
    return sf, A


def check(inst, x, nthreads: int = 0):
    rp, lits, ty, pa, _ = _inst_arrays(inst)
    x = _f64(np.atleast_2d(x))
    B = x.shape[0]
    sat = np.zeros(B, dtype=np.uint8)
    nun = np.zeros(B, dtype=np.int32)
    rc = lib().orc_check(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), B, _p(x, _dp),
                         _p(sat, _u8), _p(nun, _i32), nthreads)
    if rc != 0:
        raise ValueError("oracle: NaN or bad variable")
    return sat, nun


def step(inst, x, T: int, lr: float, seed: int = 0, epoch: int = 0, b_offset: int = 0, restart: bool = True,
         nthreads: int = 0, weights=None):
    """One round of Alg. 1 with fixed-step projected GD; returns (x_new, solved, n_unsat)."""
    rp, lits, ty, pa, w = _inst_arrays(inst)
    if weights is not None:
        w = _f64(weights)
    x = _f64(np.atleast_2d(x)).copy()
    B = x.shape[0]
    solved = np.zeros(B, dtype=np.uint8)
    nun = np.zeros(B, dtype=np.int32)
    rc = lib().orc_step(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), _p(w, _dp), B,
                        _p(x, _dp), T, lr, seed, epoch, b_offset, int(restart), _p(solved, _u8), _p(nun, _i32),
                        nthreads)
    if rc != 0:
        raise ValueError("oracle: bad input")
    return x, solved, nun


def unsat_counts(inst, x):
    rp, lits, ty, pa, _ = _inst_arrays(inst)
    x = _f64(np.atleast_2d(x))
    U = np.zeros(inst.m, dtype=np.int32)
    rc = lib().orc_unsat_counts(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), x.shape[0],
                                _p(x, _dp), _p(U, _i32))
    if rc != 0:
        raise ValueError("oracle: bad input")
    return U


def erwa(U, w, alpha: float = 0.4):
    U = np.ascontiguousarray(U, dtype=np.int32)
    w = _f64(w).copy()
    lib().orc_erwa(len(w), _p(U, _i32), alpha, _p(w, _dp))
    return w


def step_pgfp(inst, x, T: int, eta0: float, beta: float = 0.5, maxls: int = 15, eta_min: float = 1e-12,
              slack: float = 0.0, seed: int = 0, epoch: int = 0, b_offset: int = 0, restart: bool = True,
              nthreads: int = 0, weights=None):
    """One CLS round with the projected-gradient fixed-point update and FISTA
    line search (App. A.3); returns (x_new, solved, n_unsat, iterations, eta)."""
    rp, lits, ty, pa, w = _inst_arrays(inst)
    if weights is not None:
        w = _f64(weights)
    x = _f64(np.atleast_2d(x)).copy()
    B = x.shape[0]
    solved = np.zeros(B, dtype=np.uint8)
    nun = np.zeros(B, dtype=np.int32)
    its = np.zeros(B, dtype=np.int32)
    eta = np.zeros(B, dtype=np.float64)
    rc = lib().orc_step_pgfp(inst.n, inst.m, _p(rp, _i64), _p(lits, _i32), _p(ty, _u8), _p(pa, _i32), _p(w, _dp), B,
                             _p(x, _dp), T, eta0, beta, maxls, eta_min, slack, seed & 0xFFFFFFFFFFFFFFFF, epoch,
                             b_offset, int(restart), _p(solved, _u8), _p(nun, _i32), _p(its, _i32), _p(eta, _dp),
                             nthreads)
    if rc != 0:
        raise ValueError("oracle: bad input or parameters")
    return x, solved, nun, its, eta


def rephase(x, phase: int, solved=None, seed: int = 0, epoch: int = 0, b_offset: int = 0):
    """Sec. "Rephasing Heuristics": original (0), flipped (1) or random (2) phase
    for the unsolved points; returns the new points (float64)."""
    x = _f64(np.atleast_2d(x)).copy()
    s = None if solved is None else np.ascontiguousarray(solved, dtype=np.uint8)
    rc = lib().orc_rephase(x.shape[1], x.shape[0], _p(x, _dp), int(phase), None if s is None else _p(s, _u8),
                           seed & 0xFFFFFFFFFFFFFFFF, epoch, b_offset)
    if rc != 0:
        raise ValueError("oracle: unknown phase")
    return x


def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(state & 0xFFFFFFFFFFFFFFFF))


def uniform(seed: int, epoch: int, b: int, v: int) -> float:
    return lib().orc_uniform(seed, epoch, b, v)


def max_threads() -> int:
    return lib().orc_max_threads()
