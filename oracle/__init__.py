"""Naive Bayes oracle (FP64, CPU) -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and
shares no code with it.

The arithmetic lives in ``nb_oracle.c`` (plain C, FP64, rows summed with the
feature index ascending); this module compiles it with gcc, marshals numpy
arrays, and composes the steps of the paper's Sec. 4:

* fit   -- per-class counts (multinomial) or moments (Gaussian),
* joint -- s_c = log P(c) + sum_j log P(x_j | c)   (Sec. 4 equation, in logs),
* decide -- label = lowest index among the maxima (Sec. 4 decision rule, tie
  goes to benign = 0), margin = top-1 minus top-2 score, log posterior.

Storage-format helpers (what a stored u8/u16/BF16/FP8 feature value means)
are in ``oracle.formats``, written from the format definitions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``nb_oracle.c`` into ``liboracle.so`` next to it (gcc, -O2).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded on
    both x86 and Arm hosts, so the oracle gives the same bits on each.
    """
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.oracle_mn_fit.argtypes = [P, i64, i32, P, i32, f64, P, P, P, P, P]
            lib.oracle_mn_fit.restype = ctypes.c_int
            lib.oracle_mn_finalize.argtypes = [P, P, i64, i32, i32, f64, P, P, P]
            lib.oracle_mn_finalize.restype = ctypes.c_int
            lib.oracle_gauss_fit.argtypes = [P, i64, i32, P, i32, f64, P, P, P, P, P]
            lib.oracle_gauss_fit.restype = ctypes.c_int
            lib.oracle_mn_joint.argtypes = [P, i64, i32, i32, P, P, P, ctypes.c_int]
            lib.oracle_mn_joint.restype = None
            lib.oracle_gauss_joint.argtypes = [P, i64, i32, i32, P, P, P, P, ctypes.c_int]
            lib.oracle_gauss_joint.restype = None
            lib.oracle_decide.argtypes = [P, i64, i32, P, P, P]
            lib.oracle_decide.restype = None
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class OracleError(ValueError):
    pass


def mn_fit(X, y, C, alpha=1.0, log_prior=None):
    """Multinomial fit: exact uint64 counts, then FP64 log theta and log prior."""
    lib = _load()
    X = _f64(X)
    n, F = X.shape
    y = np.ascontiguousarray(y, dtype=np.int32)
    lp = None if log_prior is None else _f64(log_prior)
    counts = np.zeros((C, F), np.uint64)
    nc = np.zeros(C, np.uint64)
    log_theta = np.zeros((C, F), np.float64)
    log_pi = np.zeros(C, np.float64)
    rc = lib.oracle_mn_fit(_ptr(X), n, F, _ptr(y), C, float(alpha), _ptr(lp),
                           _ptr(counts), _ptr(nc), _ptr(log_theta), _ptr(log_pi))
    if rc != 0:
        raise OracleError("oracle_mn_fit rejected its arguments")
    return {"kind": "multinomial", "counts": counts, "nc": nc,
            "log_theta": log_theta, "log_pi": log_pi, "alpha": float(alpha)}


def mn_finalize(counts, nc, n, alpha=1.0, log_prior=None):
    """log theta and log prior from exact per-class counts (second half of mn_fit)."""
    lib = _load()
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    nc = np.ascontiguousarray(nc, dtype=np.uint64)
    C, F = counts.shape
    lp = None if log_prior is None else _f64(log_prior)
    log_theta = np.zeros((C, F), np.float64)
    log_pi = np.zeros(C, np.float64)
    rc = lib.oracle_mn_finalize(_ptr(counts), _ptr(nc), int(n), F, C, float(alpha), _ptr(lp),
                                _ptr(log_theta), _ptr(log_pi))
    if rc != 0:
        raise OracleError("oracle_mn_finalize rejected its arguments")
    return {"kind": "multinomial", "counts": counts, "nc": nc,
            "log_theta": log_theta, "log_pi": log_pi, "alpha": float(alpha)}


def gauss_fit(X, y, C, var_smoothing=1e-9, log_prior=None):
    """Gaussian fit: two-pass FP64 means and MLE variances plus epsilon."""
    lib = _load()
    X = _f64(X)
    n, F = X.shape
    y = np.ascontiguousarray(y, dtype=np.int32)
    lp = None if log_prior is None else _f64(log_prior)
    nc = np.zeros(C, np.uint64)
    mu = np.zeros((C, F), np.float64)
    var = np.zeros((C, F), np.float64)
    log_pi = np.zeros(C, np.float64)
    rc = lib.oracle_gauss_fit(_ptr(X), n, F, _ptr(y), C, float(var_smoothing),
                              _ptr(lp), _ptr(nc), _ptr(mu), _ptr(var), _ptr(log_pi))
    if rc != 0:
        raise OracleError("oracle_gauss_fit rejected its arguments")
    return {"kind": "gaussian", "nc": nc, "mu": mu, "var": var, "log_pi": log_pi}


def joint(X, model, nthreads=1):
    """Joint log scores s (n x C) for a fitted model (either kind)."""
    lib = _load()
    X = _f64(X)
    n, F = X.shape
    C = model["log_pi"].shape[0]
    s = np.zeros((n, C), np.float64)
    log_pi = _f64(model["log_pi"])
    if model["kind"] == "multinomial":
        lt = _f64(model["log_theta"])
        assert lt.shape == (C, F)
        lib.oracle_mn_joint(_ptr(X), n, F, C, _ptr(lt), _ptr(log_pi), _ptr(s),
                            int(nthreads))
    else:
        mu, var = _f64(model["mu"]), _f64(model["var"])
        assert mu.shape == (C, F) and var.shape == (C, F)
        lib.oracle_gauss_joint(_ptr(X), n, F, C, _ptr(mu), _ptr(var),
                               _ptr(log_pi), _ptr(s), int(nthreads))
    return s


def decide(s, want_lp=True):
    """Label (lowest index among maxima), top-2 margin and log posterior."""
    lib = _load()
    s = _f64(s)
    n, C = s.shape
    label = np.zeros(n, np.uint8)
    margin = np.zeros(n, np.float64)
    lp = np.zeros((n, C), np.float64) if want_lp else None
    lib.oracle_decide(_ptr(s), n, C, _ptr(label), _ptr(margin), _ptr(lp))
    return label, margin, lp


def score(X, model, nthreads=1, want_lp=True):
    """joint() then decide(): what one scoring call of the library returns."""
    s = joint(X, model, nthreads)
    label, margin, lp = decide(s, want_lp)
    return {"s": s, "label": label, "margin": margin, "lp": lp}
