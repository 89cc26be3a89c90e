"""Python binding of libffsat.so (the CUDA C-ABI library).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch tensors supply device memory and streams.  The module
fails loudly when the compiled library is missing; there is no CPU fallback.

The C entry points are reachable under their own names through ``lib()``
(``lib().ffsat_eval_grad(...)``); the ``Instance`` class wraps them for torch
tensors.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libffsat.so")

FFSAT_OR, FFSAT_XOR, FFSAT_ATLEAST = 0, 1, 2
FFSAT_F32, FFSAT_F64 = 0, 1
FFSAT_FORM_STABLE, FFSAT_FORM_PAPER = 0, 1
FFSAT_MAX_LEN = 512
FFSAT_STATIC_SCRATCH_BYTES = 32 << 20
FFSAT_PHASE_ORIGINAL, FFSAT_PHASE_FLIPPED, FFSAT_PHASE_RANDOM = 0, 1, 2

ERRORS = {
    0: "FFSAT_OK",
    -1: "FFSAT_ERR_ARG",
    -2: "FFSAT_ERR_VAR_RANGE",
    -3: "FFSAT_ERR_DUPVAR",
    -4: "FFSAT_ERR_EMPTY",
    -5: "FFSAT_ERR_PARAM",
    -6: "FFSAT_ERR_WEIGHT",
    -7: "FFSAT_ERR_TOOLONG",
    -8: "FFSAT_ERR_CUDA",
    -9: "FFSAT_ERR_NAN",
    -10: "FFSAT_ERR_DEVICE",
}

# Every symbol include/ffsat.h declares.
SYMBOLS = (
    "ffsat_default_options",
    "ffsat_load_instance",
    "ffsat_set_weights",
    "ffsat_eval_grad",
    "ffsat_eval_grad_plain64",
    "ffsat_step",
    "ffsat_step_noalloc",
    "ffsat_step_pgfp",
    "ffsat_check",
    "ffsat_unsat_counts",
    "ffsat_erwa_update",
    "ffsat_rephase",
    "ffsat_rephase_at",
    "ffsat_get_weights",
    "ffsat_batch_create",
    "ffsat_batch_eval_grad",
    "ffsat_batch_step",
    "ffsat_batch_threads",
    "ffsat_batch_free",
    "ffsat_mpnn_create",
    "ffsat_mpnn_num_params",
    "ffsat_mpnn_get_params",
    "ffsat_mpnn_set_params",
    "ffsat_mpnn_forward",
    "ffsat_mpnn_loss_grad",
    "ffsat_mpnn_adam_step",
    "ffsat_restart_from_proposal",
    "ffsat_mpnn_free",
    "ffsat_sync_status",
    "ffsat_instance_info",
    "ffsat_last_launch_count",
    "ffsat_last_cluster_size",
    "ffsat_last_points_per_cta",
    "ffsat_alu_peak",
    "ffsat_last_error",
    "ffsat_free",
)


# NVTX ranges around the library calls (for nsys / ncu timelines), enabled by
# FFSAT_NVTX=1 in the environment; off by default (no cost beyond one test).
_NVTX = os.environ.get("FFSAT_NVTX", "0") not in ("", "0")


def _traced(fn):
    if not _NVTX:
        return fn
    import functools

    @functools.wraps(fn)
    def wrapper(*a, **k):
        import torch

        torch.cuda.nvtx.range_push(f"ffsat.{fn.__qualname__}")
        try:
            return fn(*a, **k)
        finally:
            torch.cuda.nvtx.range_pop()

    return wrapper


class FFSatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("form", C.c_int32), ("node_all", C.c_int32), ("node_r", C.c_int32), ("autotune", C.c_int32),
                ("device", C.c_int32), ("cluster", C.c_int32)]


class StepArgs(C.Structure):
    _fields_ = [("T", C.c_int32), ("restart", C.c_int32), ("lr", C.c_double), ("seed", C.c_uint64),
                ("epoch", C.c_uint64), ("b_offset", C.c_uint64), ("unsat_counts", C.c_void_p)]


class PgfpArgs(C.Structure):
    _fields_ = [("T", C.c_int32), ("restart", C.c_int32), ("eta0", C.c_double), ("beta", C.c_double),
                ("maxls", C.c_int32), ("pad", C.c_int32), ("eta_min", C.c_double), ("slack", C.c_double),
                ("seed", C.c_uint64), ("epoch", C.c_uint64), ("b_offset", C.c_uint64),
                ("unsat_counts", C.c_void_p), ("iters", C.c_void_p), ("eta_out", C.c_void_p)]


class BatchIO(C.Structure):
    _fields_ = [("B", C.c_int32), ("pad", C.c_int32), ("x", C.c_void_p), ("f", C.c_void_p), ("g", C.c_void_p),
                ("solved", C.c_void_p), ("n_unsat", C.c_void_p), ("b_offset", C.c_uint64)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int64), ("n_clause3", C.c_int32),
                ("n_product", C.c_int32), ("n_node", C.c_int32), ("n_const", C.c_int32), ("n_tables", C.c_int32),
                ("n_tasks", C.c_int32), ("node_r", C.c_int32), ("smem_mode_f32", C.c_int32),
                ("smem_mode_f64", C.c_int32), ("threads_f32", C.c_int32), ("node_lane_work", C.c_int64),
                ("device_bytes", C.c_int64), ("autotuned", C.c_int32), ("autotune_us", C.c_float * 2),
                ("n_xor2", C.c_int32), ("pad", C.c_int32), ("smem_bytes_f32", C.c_int64),
                ("smem_bytes_f64", C.c_int64), ("tune_shape", C.c_int32), ("tune_clause_k", C.c_int32),
                ("tune_pts_per_cta", C.c_int32), ("tune_candidates", C.c_int32), ("tune_cached", C.c_int32),
                ("fix_words_f32", C.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["autotune_us"] = list(self.autotune_us)
        return d


_lib = None
_vp = C.c_void_p


def lib():
    """Load libffsat.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(
                f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                "or `python paper_2308_15020_gb300/build.py`")
        L = C.CDLL(LIB_PATH)
        L.ffsat_default_options.argtypes = [C.POINTER(Options)]
        L.ffsat_default_options.restype = None
        L.ffsat_load_instance.argtypes = [C.c_int32, C.c_int32, _vp, _vp, _vp, _vp, _vp, C.POINTER(Options),
                                          C.POINTER(_vp)]
        L.ffsat_load_instance.restype = C.c_int
        L.ffsat_set_weights.argtypes = [_vp, _vp]
        L.ffsat_set_weights.restype = C.c_int
        L.ffsat_eval_grad.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
        L.ffsat_eval_grad.restype = C.c_int
        L.ffsat_eval_grad_plain64.argtypes = [_vp, C.c_int32, _vp, _vp, _vp, _vp]
        L.ffsat_eval_grad_plain64.restype = C.c_int
        L.ffsat_step.argtypes = [_vp, C.c_int32, _vp, C.c_int32, C.POINTER(StepArgs), _vp, _vp, _vp]
        L.ffsat_step.restype = C.c_int
        L.ffsat_step_noalloc.argtypes = [_vp, C.c_int32, _vp, C.c_int32, C.POINTER(StepArgs), _vp, _vp, _vp]
        L.ffsat_step_noalloc.restype = C.c_int
        L.ffsat_step_pgfp.argtypes = [_vp, C.c_int32, _vp, C.c_int32, C.POINTER(PgfpArgs), _vp, _vp, _vp]
        L.ffsat_step_pgfp.restype = C.c_int
        L.ffsat_check.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp]
        L.ffsat_check.restype = C.c_int
        L.ffsat_unsat_counts.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, _vp]
        L.ffsat_unsat_counts.restype = C.c_int
        L.ffsat_erwa_update.argtypes = [_vp, _vp, C.c_double, _vp]
        L.ffsat_erwa_update.restype = C.c_int
        L.ffsat_rephase.argtypes = [_vp, C.c_int32, _vp, C.c_int32, C.c_int32, _vp, C.c_uint64, C.c_uint64,
                                    C.c_uint64, _vp]
        L.ffsat_rephase.restype = C.c_int
        L.ffsat_rephase_at.argtypes = [_vp, C.c_int32, _vp, C.c_int32, C.c_int32, _vp, C.c_uint64, _vp,
                                       C.c_uint64, _vp]
        L.ffsat_rephase_at.restype = C.c_int
        L.ffsat_get_weights.argtypes = [_vp, _vp]
        L.ffsat_get_weights.restype = C.c_int
        L.ffsat_batch_create.argtypes = [C.POINTER(_vp), C.c_int32, C.POINTER(_vp)]
        L.ffsat_batch_create.restype = C.c_int
        L.ffsat_batch_eval_grad.argtypes = [_vp, C.POINTER(BatchIO), C.c_int32, _vp]
        L.ffsat_batch_eval_grad.restype = C.c_int
        L.ffsat_batch_step.argtypes = [_vp, C.POINTER(BatchIO), C.c_int32, C.POINTER(StepArgs), _vp]
        L.ffsat_batch_step.restype = C.c_int
        L.ffsat_batch_threads.argtypes = [_vp, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_float),
                                          C.POINTER(C.c_float)]
        L.ffsat_batch_threads.restype = C.c_int
        L.ffsat_batch_free.argtypes = [_vp]
        L.ffsat_batch_free.restype = None
        L.ffsat_mpnn_create.argtypes = [C.c_int32, C.c_uint64, C.POINTER(_vp)]
        L.ffsat_mpnn_create.restype = C.c_int
        L.ffsat_mpnn_num_params.argtypes = [_vp]
        L.ffsat_mpnn_num_params.restype = C.c_int32
        L.ffsat_mpnn_get_params.argtypes = [_vp, _vp]
        L.ffsat_mpnn_get_params.restype = C.c_int
        L.ffsat_mpnn_set_params.argtypes = [_vp, _vp]
        L.ffsat_mpnn_set_params.restype = C.c_int
        L.ffsat_mpnn_forward.argtypes = [_vp, _vp, _vp, _vp]
        L.ffsat_mpnn_forward.restype = C.c_int
        L.ffsat_mpnn_loss_grad.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.ffsat_mpnn_loss_grad.restype = C.c_int
        L.ffsat_mpnn_adam_step.argtypes = [_vp, C.c_float, _vp]
        L.ffsat_mpnn_adam_step.restype = C.c_int
        L.ffsat_restart_from_proposal.argtypes = [_vp, C.c_int32, _vp, C.c_int32, _vp, C.c_float, _vp, C.c_uint64,
                                                  C.c_uint64, C.c_uint64, _vp]
        L.ffsat_restart_from_proposal.restype = C.c_int
        L.ffsat_alu_peak.argtypes = [C.c_int32, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]
        L.ffsat_alu_peak.restype = C.c_int
        L.ffsat_mpnn_free.argtypes = [_vp]
        L.ffsat_mpnn_free.restype = None
        L.ffsat_sync_status.argtypes = [_vp, _vp]
        L.ffsat_sync_status.restype = C.c_int
        L.ffsat_instance_info.argtypes = [_vp, C.POINTER(Info)]
        L.ffsat_instance_info.restype = C.c_int
        L.ffsat_last_launch_count.argtypes = []
        L.ffsat_last_launch_count.restype = C.c_int32
        L.ffsat_last_cluster_size.argtypes = []
        L.ffsat_last_cluster_size.restype = C.c_int32
        L.ffsat_last_points_per_cta.argtypes = []
        L.ffsat_last_points_per_cta.restype = C.c_int32
        L.ffsat_last_error.argtypes = []
        L.ffsat_last_error.restype = C.c_char_p
        L.ffsat_free.argtypes = [_vp]
        L.ffsat_free.restype = None
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise FFSatError(rc, lib().ffsat_last_error().decode())


def last_launch_count() -> int:
    return int(lib().ffsat_last_launch_count())


def last_cluster_size() -> int:
    """CTAs per point of the last step call on this thread (1: one CTA per point)."""
    return int(lib().ffsat_last_cluster_size())


def last_points_per_cta() -> int:
    """Points per CTA of the last step call on this thread (2: two points per CTA)."""
    return int(lib().ffsat_last_points_per_cta())


def alu_peak(dtype: int = FFSAT_F32, target_ms: float = 50.0, stream=None):
    """Measured FMA throughput of the current device (TFLOP/s) and the timed
    launch's duration (ms): FFSAT_F32 or FFSAT_F64."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    _check(lib().ffsat_alu_peak(int(dtype), float(target_ms), C.byref(tf), C.byref(ms), _stream(stream)))
    return tf.value, ms.value


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dtype_code(t) -> int:
    import torch

    if t.dtype == torch.float32:
        return FFSAT_F32
    if t.dtype == torch.float64:
        return FFSAT_F64
    raise TypeError(f"x must be float32 or float64, got {t.dtype}")


def _need_cuda_contig(t, name):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


class Instance:
    """An instance loaded into the library (``ffsat_load_instance``)."""

    def __init__(self, inst, form: int = FFSAT_FORM_STABLE, node_all: bool = False, node_r: int = 0,
                 autotune: bool = False, device: int = -1, cluster: int = 0):
        import numpy as np

        self.n = int(inst.n)
        self.m = int(inst.ctype.shape[0])
        self._rp = np.ascontiguousarray(inst.row_ptr, dtype=np.int64)
        self._lits = np.ascontiguousarray(inst.lits, dtype=np.int32)
        self._ty = np.ascontiguousarray(inst.ctype, dtype=np.uint8)
        self._pa = np.ascontiguousarray(inst.param, dtype=np.int32)
        self._w = np.ascontiguousarray(inst.weights, dtype=np.float64)
        opt = Options()
        lib().ffsat_default_options(C.byref(opt))
        opt.form, opt.node_all, opt.node_r, opt.autotune, opt.device = form, int(node_all), node_r, int(autotune), device
        opt.cluster = cluster
        h = _vp()
        rc = lib().ffsat_load_instance(self.n, self.m, self._rp.ctypes.data, self._lits.ctypes.data,
                                       self._ty.ctypes.data, self._pa.ctypes.data, self._w.ctypes.data,
                                       C.byref(opt), C.byref(h))
        _check(rc)
        self.handle = h.value

    # -- lifetime --------------------------------------------------------------------------
    def free(self):
        if getattr(self, "handle", None):
            lib().ffsat_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        inf = Info()
        _check(lib().ffsat_instance_info(self.handle, C.byref(inf)))
        return inf.as_dict()

    @_traced
    def set_weights(self, w):
        import numpy as np

        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (self.m,):
            raise ValueError("weights must have shape (m,)")
        _check(lib().ffsat_set_weights(self.handle, w.ctypes.data))
        self._w = w

    @property
    def host_weights(self):
        """The weights last given at load or to set_weights (ERWA updates live on the device)."""
        return self._w

    # -- hot path ----------------------------------------------------------------------------
    @_traced
    def eval_grad(self, x, f=None, g=None, want_f: bool = True, want_g: bool = True, stream=None):
        """f[b] = F(x_b) (float64) and g = grad F (dtype of x)."""
        import torch

        _need_cuda_contig(x, "x")
        B = x.shape[0]
        if want_f and f is None:
            f = torch.empty(B, dtype=torch.float64, device=x.device)
        if want_g and g is None:
            g = torch.empty_like(x)
        rc = lib().ffsat_eval_grad(self.handle, B, x.data_ptr(), _dtype_code(x), _ptr(f if want_f else None),
                                   _ptr(g if want_g else None), _stream(stream))
        _check(rc)
        return f, g

    @_traced
    def eval_grad_plain64(self, x, f=None, g=None, stream=None):
        import torch

        _need_cuda_contig(x, "x")
        if x.dtype != torch.float64:
            raise TypeError("the plain FP64 path takes float64 x")
        B = x.shape[0]
        f = torch.empty(B, dtype=torch.float64, device=x.device) if f is None else f
        g = torch.empty_like(x) if g is None else g
        _check(lib().ffsat_eval_grad_plain64(self.handle, B, x.data_ptr(), f.data_ptr(), g.data_ptr(),
                                             _stream(stream)))
        return f, g

    @_traced
    def step(self, x, T: int, lr: float, seed: int = 0, epoch: int = 0, b_offset: int = 0, restart: bool = True,
             solved=None, n_unsat=None, unsat_counts=None, stream=None):
        """One round of fixed-step projected GD + exact check + restart, in place on x.
        With ``unsat_counts`` (int32 [m], zeroed by the caller) the check also adds
        the per-constraint violation counts of the final points."""
        import torch

        _need_cuda_contig(x, "x")
        B = x.shape[0]
        if solved is None:
            solved = torch.empty(B, dtype=torch.uint8, device=x.device)
        if n_unsat is None:
            n_unsat = torch.empty(B, dtype=torch.int32, device=x.device)
        a = StepArgs(int(T), int(restart), float(lr), int(seed) & (2**64 - 1), int(epoch), int(b_offset),
                     _ptr(self._counts_arg(unsat_counts)))
        _check(lib().ffsat_step(self.handle, B, x.data_ptr(), _dtype_code(x), C.byref(a), solved.data_ptr(),
                                n_unsat.data_ptr(), _stream(stream)))
        return solved, n_unsat

    @_traced
    def step_noalloc(self, x, T: int, lr: float, seed: int = 0, epoch: int = 0, b_offset: int = 0,
                     restart: bool = True, solved=None, n_unsat=None, unsat_counts=None, stream=None):
        """``step`` through ``ffsat_step_noalloc``: no device allocation, static scratch."""
        import torch

        _need_cuda_contig(x, "x")
        B = x.shape[0]
        if solved is None:
            solved = torch.empty(B, dtype=torch.uint8, device=x.device)
        if n_unsat is None:
            n_unsat = torch.empty(B, dtype=torch.int32, device=x.device)
        a = StepArgs(int(T), int(restart), float(lr), int(seed) & (2**64 - 1), int(epoch), int(b_offset),
                     _ptr(self._counts_arg(unsat_counts)))
        _check(lib().ffsat_step_noalloc(self.handle, B, x.data_ptr(), _dtype_code(x), C.byref(a), solved.data_ptr(),
                                        n_unsat.data_ptr(), _stream(stream)))
        return solved, n_unsat

    @_traced
    def step_pgfp(self, x, T: int, eta0: float, beta: float = 0.5, maxls: int = 15, eta_min: float = 1e-12,
                  slack: Optional[float] = None, seed: int = 0, epoch: int = 0, b_offset: int = 0,
                  restart: bool = True, solved=None, n_unsat=None, unsat_counts=None, iters=None, eta_out=None,
                  stream=None):
        """One round of projected gradient with FISTA line search (``ffsat_step_pgfp``).
        slack defaults to 1e-6 (FP32) or 0 (FP64) times the sum of the host weights."""
        import torch

        _need_cuda_contig(x, "x")
        B = x.shape[0]
        if solved is None:
            solved = torch.empty(B, dtype=torch.uint8, device=x.device)
        if n_unsat is None:
            n_unsat = torch.empty(B, dtype=torch.int32, device=x.device)
        if slack is None:
            slack = (1e-6 if x.dtype == torch.float32 else 0.0) * float(self._w.sum())
        a = PgfpArgs(int(T), int(restart), float(eta0), float(beta), int(maxls), 0, float(eta_min), float(slack),
                     int(seed) & (2**64 - 1), int(epoch), int(b_offset), _ptr(self._counts_arg(unsat_counts)),
                     _ptr(iters), _ptr(eta_out))
        _check(lib().ffsat_step_pgfp(self.handle, B, x.data_ptr(), _dtype_code(x), C.byref(a), solved.data_ptr(),
                                     n_unsat.data_ptr(), _stream(stream)))
        return solved, n_unsat

    @_traced
    def check(self, x, sat=None, n_unsat=None, stream=None):
        import torch

        _need_cuda_contig(x, "x")
        B = x.shape[0]
        sat = torch.empty(B, dtype=torch.uint8, device=x.device) if sat is None else sat
        n_unsat = torch.empty(B, dtype=torch.int32, device=x.device) if n_unsat is None else n_unsat
        _check(lib().ffsat_check(self.handle, B, x.data_ptr(), _dtype_code(x), sat.data_ptr(), n_unsat.data_ptr(),
                                 _stream(stream)))
        return sat, n_unsat

    def sync_status(self, stream=None):
        _check(lib().ffsat_sync_status(self.handle, _stream(stream)))

    # -- restart heuristics ------------------------------------------------------------------
    def _counts_arg(self, U):
        if U is None:
            return None
        import torch

        _need_cuda_contig(U, "unsat_counts")
        if U.dtype != torch.int32 or U.numel() != self.m:
            raise ValueError("unsat_counts must be an int32 tensor of m elements")
        return U

    @_traced
    def unsat_counts(self, x, U=None, stream=None):
        """U[c] = number of points of x whose sign vector violates constraint c."""
        import torch

        _need_cuda_contig(x, "x")
        U = torch.empty(self.m, dtype=torch.int32, device=x.device) if U is None else self._counts_arg(U)
        _check(lib().ffsat_unsat_counts(self.handle, x.shape[0], x.data_ptr(), _dtype_code(x), _ptr(U),
                                        _stream(stream)))
        return U

    @_traced
    def erwa_update(self, U, alpha: float = 0.4, stream=None):
        """Device ERWA update w <- (1 - alpha) w + alpha U / max U of every weight."""
        _check(lib().ffsat_erwa_update(self.handle, _ptr(self._counts_arg(U)), float(alpha), _stream(stream)))

    @_traced
    def rephase(self, x, phase: int, solved=None, seed: int = 0, epoch: int = 0, b_offset: int = 0, stream=None,
                epoch_dev=None):
        """Original (0) / flipped (1) / random (2) phase for the unsolved points of x, in place.
        With epoch_dev (a one-element int64 device tensor) the epoch is read on the device."""
        _need_cuda_contig(x, "x")
        if epoch_dev is not None:
            _check(lib().ffsat_rephase_at(self.handle, x.shape[0], x.data_ptr(), _dtype_code(x), int(phase),
                                          _ptr(solved), int(seed) & (2**64 - 1), epoch_dev.data_ptr(),
                                          int(b_offset), _stream(stream)))
            return x
        _check(lib().ffsat_rephase(self.handle, x.shape[0], x.data_ptr(), _dtype_code(x), int(phase), _ptr(solved),
                                   int(seed) & (2**64 - 1), int(epoch), int(b_offset), _stream(stream)))
        return x

    def get_weights(self):
        import numpy as np

        w = np.empty(self.m, dtype=np.float64)
        _check(lib().ffsat_get_weights(self.handle, w.ctypes.data))
        return w


class Batch:
    """Several loaded instances evaluated in one launch (``ffsat_batch_*``)."""

    def __init__(self, instances):
        self.instances = list(instances)  # keep them alive
        arr = (_vp * len(self.instances))(*[h.handle for h in self.instances])
        h = _vp()
        _check(lib().ffsat_batch_create(arr, len(self.instances), C.byref(h)))
        self.handle = h.value

    def free(self):
        if getattr(self, "handle", None):
            lib().ffsat_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def threads(self, dtype: int = FFSAT_F32):
        """(threads per CTA of the batch kernel, FP32 probe times at 384 and 512 threads in us)."""
        th, a, b = C.c_int32(0), C.c_float(0.0), C.c_float(0.0)
        _check(lib().ffsat_batch_threads(self.handle, int(dtype), C.byref(th), C.byref(a), C.byref(b)))
        return th.value, a.value, b.value

    def _io(self, xs, fs=None, gs=None, solved=None, n_unsat=None, b_offsets=None):
        io = (BatchIO * len(self.instances))()
        dt = None
        for k, x in enumerate(xs):
            _need_cuda_contig(x, f"xs[{k}]")
            d = _dtype_code(x)
            if dt is not None and d != dt:
                raise TypeError("all x must share one dtype")
            dt = d
            io[k].B = x.shape[0]
            io[k].x = x.data_ptr()
            io[k].f = _ptr(fs[k]) if fs else None
            io[k].g = _ptr(gs[k]) if gs else None
            io[k].solved = _ptr(solved[k]) if solved else None
            io[k].n_unsat = _ptr(n_unsat[k]) if n_unsat else None
            io[k].b_offset = int(b_offsets[k]) if b_offsets is not None else 0
        return io, dt

    @_traced
    def eval_grad(self, xs, fs=None, gs=None, stream=None):
        import torch

        if fs is None:
            fs = [torch.empty(x.shape[0], dtype=torch.float64, device=x.device) for x in xs]
        if gs is None:
            gs = [torch.empty_like(x) for x in xs]
        io, dt = self._io(xs, fs, gs)
        _check(lib().ffsat_batch_eval_grad(self.handle, io, dt, _stream(stream)))
        return fs, gs

    @_traced
    def step(self, xs, T: int, lr: float, seed: int = 0, epoch: int = 0, restart: bool = True, b_offsets=None,
             solved=None, n_unsat=None, stream=None):
        import torch

        if solved is None:
            solved = [torch.empty(x.shape[0], dtype=torch.uint8, device=x.device) for x in xs]
        if n_unsat is None:
            n_unsat = [torch.empty(x.shape[0], dtype=torch.int32, device=x.device) for x in xs]
        io, dt = self._io(xs, solved=solved, n_unsat=n_unsat, b_offsets=b_offsets)
        a = StepArgs(int(T), int(restart), float(lr), int(seed) & (2**64 - 1), int(epoch), 0)
        _check(lib().ffsat_batch_step(self.handle, io, dt, C.byref(a), _stream(stream)))
        return solved, n_unsat


class MPNN:
    """The learned restart proposal network (``ffsat_mpnn_*``)."""

    def __init__(self, layers: int = 3, seed: int = 0):
        h = _vp()
        _check(lib().ffsat_mpnn_create(int(layers), int(seed) & (2**64 - 1), C.byref(h)))
        self.handle = h.value
        self.layers = layers

    def free(self):
        if getattr(self, "handle", None):
            lib().ffsat_mpnn_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def num_params(self) -> int:
        return int(lib().ffsat_mpnn_num_params(self.handle))

    def get_params(self):
        import numpy as np

        p = np.zeros(self.num_params(), dtype=np.float32)
        _check(lib().ffsat_mpnn_get_params(self.handle, p.ctypes.data))
        return p

    def set_params(self, p):
        import numpy as np

        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.shape != (self.num_params(),):
            raise ValueError("wrong parameter count")
        _check(lib().ffsat_mpnn_set_params(self.handle, p.ctypes.data))

    def forward(self, inst: Instance, x0=None, stream=None):
        import torch

        if x0 is None:
            x0 = torch.empty(inst.n, dtype=torch.float32, device="cuda")
        _check(lib().ffsat_mpnn_forward(self.handle, inst.handle, x0.data_ptr(), _stream(stream)))
        return x0

    def loss_grad(self, inst: Instance, target, loss=None, x0=None, want_host_grad: bool = False, stream=None):
        """(loss tensor, proposal tensor, host gradient or None)."""
        import numpy as np
        import torch

        _need_cuda_contig(target, "target")
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        if x0 is None:
            x0 = torch.empty(inst.n, dtype=torch.float32, device="cuda")
        gh = np.zeros(self.num_params(), dtype=np.float32) if want_host_grad else None
        _check(lib().ffsat_mpnn_loss_grad(self.handle, inst.handle, target.data_ptr(), loss.data_ptr(), x0.data_ptr(),
                                          None if gh is None else gh.ctypes.data, _stream(stream)))
        return loss, x0, gh

    def adam_step(self, lr: float, stream=None):
        _check(lib().ffsat_mpnn_adam_step(self.handle, float(lr), _stream(stream)))


def restart_from_proposal(inst: Instance, x, proposal, noise: float, solved=None, seed: int = 0, epoch: int = 0,
                          b_offset: int = 0, stream=None):
    _need_cuda_contig(x, "x")
    _check(lib().ffsat_restart_from_proposal(inst.handle, x.shape[0], x.data_ptr(), _dtype_code(x), proposal.data_ptr(),
                                             float(noise), _ptr(solved), int(seed) & (2**64 - 1), int(epoch),
                                             int(b_offset), _stream(stream)))


def load_instance(inst, **kw) -> Instance:
    return Instance(inst, **kw)
