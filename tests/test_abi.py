"""The C-ABI library loads, exports every symbol include/ffsat.h declares, and
rejects malformed instances before touching the device (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2308_15020_gb300 import build, ffsat

    build.build()
    ffsat.lib()
    return ffsat


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ffsat.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ffsat_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(F):
    decl = declared_symbols()
    assert len(decl) >= 12
    L = C.CDLL(F.LIB_PATH)
    for s in decl:
        assert hasattr(L, s), s
    assert sorted(F.SYMBOLS) == decl


def test_default_options(F):
    o = F.Options()
    F.lib().ffsat_default_options(C.byref(o))
    assert (o.form, o.node_all, o.node_r, o.autotune, o.device, o.cluster) == (0, 0, 0, 0, -1, 0)


def _load(F, n, rp, lits, ty, pa, w=None, **opt):
    o = F.Options()
    F.lib().ffsat_default_options(C.byref(o))
    for k, v in opt.items():
        setattr(o, k, v)
    rp = np.asarray(rp, np.int64)
    lits = np.asarray(lits, np.int32)
    ty = np.asarray(ty, np.uint8)
    pa = np.asarray(pa, np.int32)
    wp = None if w is None else np.asarray(w, np.float64)
    h = C.c_void_p()
    rc = F.lib().ffsat_load_instance(n, len(ty), rp.ctypes.data, lits.ctypes.data if lits.size else None,
                                     ty.ctypes.data if ty.size else None, pa.ctypes.data if pa.size else None,
                                     None if wp is None else wp.ctypes.data, C.byref(o), C.byref(h))
    msg = F.lib().ffsat_last_error().decode()
    if rc == 0:
        F.lib().ffsat_free(h)
    return rc, msg


@pytest.mark.parametrize("case,code", [
    (dict(n=0, rp=[0, 1], lits=[1], ty=[0], pa=[0]), -1),                    # no variables
    (dict(n=3, rp=[0, 2], lits=[1, 4], ty=[0], pa=[0]), -2),                 # variable out of range
    (dict(n=3, rp=[0, 2], lits=[1, 0], ty=[0], pa=[0]), -2),                 # literal 0
    (dict(n=3, rp=[0, 2], lits=[2, -2], ty=[0], pa=[0]), -3),                # duplicate variable
    (dict(n=3, rp=[0, 0], lits=[], ty=[2], pa=[1]), -4),                     # empty constraint
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[7], pa=[0]), -5),                 # unknown type
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[1], pa=[2]), -5),                 # parity not 0/1
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[2], pa=[-1]), -5),                # K < 0
    (dict(n=3, rp=[1, 2], lits=[1, 2], ty=[0], pa=[0]), -5),                 # row_ptr[0] != 0
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[0], pa=[0], w=[-1.0]), -6),       # negative weight
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[0], pa=[0], w=[np.inf]), -6),     # non-finite weight
    (dict(n=600, rp=[0, 513], lits=list(range(1, 514)), ty=[2], pa=[3]), -7),  # longer than 512
    (dict(n=100, rp=[0, 61], lits=list(range(1, 62)), ty=[2], pa=[3], form=1), -7),  # paper form > 60
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[0], pa=[0], node_r=5), -1),        # bad option
    (dict(n=3, rp=[0, 2], lits=[1, 2], ty=[0], pa=[0], cluster=3), -1),       # cluster size not 0/1/2/4/8
])
def test_validation_codes(F, case, code):
    rc, msg = _load(F, case.pop("n"), case.pop("rp"), case.pop("lits"), case.pop("ty"), case.pop("pa"),
                    case.pop("w", None), **case)
    assert rc == code, msg
    assert msg


def test_valid_instance_needs_a_device(F):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    rc, msg = _load(F, 3, [0, 2], [1, -2], [0], [0])
    assert rc == -8 and "cuda" in msg.lower()


def test_missing_library_fails_loudly(monkeypatch):
    from paper_2308_15020_gb300 import ffsat

    monkeypatch.setattr(ffsat, "_lib", None)
    monkeypatch.setattr(ffsat, "LIB_PATH", "/nonexistent/libffsat.so")
    with pytest.raises(FileNotFoundError):
        ffsat.lib()


def test_null_instance_is_an_argument_error(F):
    """Every entry point that takes an instance rejects NULL with FFSAT_ERR_ARG
    before touching the device."""
    L = F.lib()
    a = F.StepArgs(1, 0, 0.1, 0, 0, 0, None)
    pa = F.PgfpArgs(1, 0, 0.1, 0.5, 4, 0, 1e-12, 0.0, 0, 0, 0, None, None, None)
    w = np.zeros(4)
    calls = {
        "ffsat_set_weights": lambda: L.ffsat_set_weights(None, w.ctypes.data),
        "ffsat_eval_grad": lambda: L.ffsat_eval_grad(None, 1, None, 0, None, None, None),
        "ffsat_eval_grad_plain64": lambda: L.ffsat_eval_grad_plain64(None, 1, None, None, None, None),
        "ffsat_step": lambda: L.ffsat_step(None, 1, None, 0, C.byref(a), None, None, None),
        "ffsat_step_noalloc": lambda: L.ffsat_step_noalloc(None, 1, None, 0, C.byref(a), None, None, None),
        "ffsat_step_pgfp": lambda: L.ffsat_step_pgfp(None, 1, None, 0, C.byref(pa), None, None, None),
        "ffsat_check": lambda: L.ffsat_check(None, 1, None, 0, None, None, None),
        "ffsat_unsat_counts": lambda: L.ffsat_unsat_counts(None, 1, None, 0, None, None),
        "ffsat_erwa_update": lambda: L.ffsat_erwa_update(None, None, 0.4, None),
        "ffsat_rephase": lambda: L.ffsat_rephase(None, 1, None, 0, 1, None, 0, 0, 0, None),
        "ffsat_get_weights": lambda: L.ffsat_get_weights(None, w.ctypes.data),
        "ffsat_restart_from_proposal": lambda: L.ffsat_restart_from_proposal(None, 1, None, 0, None, 0.5, None, 0, 0,
                                                                            0, None),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert F.lib().ffsat_last_error().decode(), name
