"""nbgpu: Naive Bayes fit and group scoring on one sm_103a GPU.

Thin Python binding over the C ABI of ``libnbgpu.so`` (declared in
``include/nbgpu.h``).  This module only marshals arguments: every step of
the fit and of the scoring runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams.  If the library is missing the import of
the entry points fails loudly -- there is no CPU fallback.

Low-level names mirror the C functions (``nb_fit``, ``nb_score_group`` ...)
and take raw device pointers; ``fit`` / ``score`` / ``Model`` accept torch
tensors.  Method: Sahay & Chaudhari, Sec. 4 (posterior and decision rule).
"""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB, build  # noqa: F401

# ---- enums (nbgpu.h) -------------------------------------------------------
NB_OK, NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ETIMEOUT, NB_EUNSUPPORTED, NB_EBUSY = range(7)
NB_MULTINOMIAL, NB_GAUSSIAN = 0, 1
NB_F32, NB_U16, NB_U8, NB_BF16, NB_FP8E4M3 = range(5)
NB_RECHECK_OFF, NB_RECHECK_LABEL, NB_RECHECK_LP = 0, 1, 2

STATUS_NAMES = {0: "NB_OK", 1: "NB_EINVAL", 2: "NB_ENOMEM", 3: "NB_ECUDA",
                4: "NB_ETIMEOUT", 5: "NB_EUNSUPPORTED", 6: "NB_EBUSY"}

_P = ctypes.c_void_p
_i32, _i64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double


class NbAux(ctypes.Structure):
    _fields_ = [("ovf_ptr", _P), ("ovf_col", _P), ("ovf_add", _P), ("row_exp", _P)]


class NbFitOpts(ctypes.Structure):
    _fields_ = [("alpha", _f64), ("log_prior", _P), ("var_smoothing", _f64),
                ("aux", ctypes.POINTER(NbAux)), ("no_sync", ctypes.c_int)]


class NbScoreOpts(ctypes.Structure):
    _fields_ = [("want_logpost", ctypes.c_int), ("recheck", ctypes.c_int),
                ("aux", ctypes.POINTER(NbAux))]


class NbTileConfig(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("stages", ctypes.c_int),
                ("rows_per_stage", ctypes.c_int), ("rows_per_warp", ctypes.c_int)]


NB_VARIANT_AUTO, NB_VARIANT_PIPELINED, NB_VARIANT_REGISTER = 0, 1, 2
NB_PATH_TWO_CLASS, NB_PATH_TENSOR, NB_PATH_TENSOR_GAUSS, NB_PATH_GENERAL = 0, 1, 2, 3
NB_SELECT_TOTAL, NB_SELECT_FILES = 0, 1
ST_BAD_ROUTE = 32          # status bit of nb_route / nb_gather / nb_groupwise_status


class NbGroup(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("X", _P), ("n", _i64), ("ld", _i64), ("aux", NbAux),
                ("label", _P), ("margin", _P), ("logpost", _P)]


class NbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes)
_SIGS = [
    ("nb_fit", ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, _i64, _i32, _i64, _P, _i32,
                              ctypes.POINTER(NbFitOpts), _P, ctypes.POINTER(_P)]),
    ("nb_refit", ctypes.c_int, [_P, _P, ctypes.c_int, _i64, _i64, _P,
                                ctypes.POINTER(NbFitOpts), _P]),
    ("nb_refit_gaussian_noalloc", ctypes.c_int, [_P, _P, _i64, _i64, _P,
                                                 ctypes.POINTER(NbFitOpts), _P]),
    ("nb_model_check", ctypes.c_int, [_P]),
    ("nb_model_counts", ctypes.c_int, [_P, _P, _P]),
    ("nb_model_params", ctypes.c_int, [_P, _P, _P, _P]),
    ("nb_model_info", ctypes.c_int, [_P, _P, _P, _P]),
    ("nb_model_free", None, [_P]),
    ("nb_score_group", ctypes.c_int, [_P, _P, ctypes.c_int, _i64, _i64, _P, _P, _P,
                                      ctypes.POINTER(NbScoreOpts), _P, _P]),
    ("nb_set_tile_config", ctypes.c_int, [_P, ctypes.POINTER(NbTileConfig)]),
    ("nb_get_tile_config", ctypes.c_int, [_P, ctypes.POINTER(NbTileConfig)]),
    ("nb_autotune_score", ctypes.c_int, [_P, _P, ctypes.c_int, _i64, _i64,
                                         ctypes.POINTER(NbAux), _P,
                                         ctypes.POINTER(NbTileConfig),
                                         ctypes.POINTER(ctypes.c_float)]),
    ("nb_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, _i64,
                                       ctypes.c_int, ctypes.POINTER(NbScoreOpts),
                                       ctypes.POINTER(_P)]),
    ("nb_batch_score", ctypes.c_int, [_P, ctypes.POINTER(NbGroup), ctypes.c_int, _P, _P]),
    ("nb_batch_capture", ctypes.c_int, [_P, _P]),
    ("nb_batch_destroy", None, [_P]),
    ("nb_server_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_size_t, ctypes.c_int,
                                        ctypes.POINTER(NbScoreOpts), ctypes.POINTER(_P)]),
    ("nb_classify_stream", ctypes.c_int, [_P, ctypes.c_int, _P, _i64, _i32, _P, _P, _P,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("nb_classify_stream_batch", ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P,
                                                _P, ctypes.POINTER(ctypes.c_int)]),
    ("nb_clock_us", ctypes.c_double, []),
    ("nb_wait", ctypes.c_int, [_P, ctypes.c_uint64, _i64]),
    ("nb_server_stats", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    ("nb_server_destroy", None, [_P]),
    ("nb_pack_u8_count", ctypes.c_int, [_P, _i64, _i32, _i64, _P, ctypes.POINTER(_i64), _P]),
    ("nb_pack_u8_fill", ctypes.c_int, [_P, _i64, _i32, _i64, _P, _i64, _P, _P, _P, _P]),
    ("nb_pack_bf16", ctypes.c_int, [_P, ctypes.c_int, _i64, _i32, _i64, _P, _i64, _P]),
    ("nb_pack_fp8", ctypes.c_int, [_P, ctypes.c_int, _i64, _i32, _i64, _P, _i64, _P, _P]),
    ("nb_group_fallback", ctypes.c_int, [_P, _i32, _i32, _i64, _P]),
    ("nb_route_workspace", ctypes.c_size_t, [_i64, _i32]),
    ("nb_route", ctypes.c_int, [_P, _i64, _i64, _i32, _P, _i32, _P, _i32, _P, _P, _P, _P, _P,
                                ctypes.c_size_t, _P, _P]),
    ("nb_select_features", ctypes.c_int, [ctypes.POINTER(_P), _i32, _i32, _i32, _P, _P]),
    ("nb_gather", ctypes.c_int, [_P, ctypes.c_int, _i64, _i32, _i64, _i64, _P, _P, _i32, _P,
                                 _i32, _P, _i64, _P, _P]),
    ("nb_groupwise_create", ctypes.c_int, [ctypes.POINTER(_P), _i32, _P, _i32, _P, _i32, _i64,
                                           _i32, ctypes.c_int, _i64,
                                           ctypes.POINTER(NbScoreOpts), ctypes.POINTER(_P)]),
    ("nb_groupwise_classify", ctypes.c_int, [_P, _P, _i64, _P, _i64, _P, _P, _P, _P, _P]),
    ("nb_groupwise_status", ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    ("nb_groupwise_destroy", None, [_P]),
    ("nb_score_path", ctypes.c_int, [_P, _P, ctypes.c_int, _i64, ctypes.c_int]),
    ("nb_last_error", ctypes.c_char_p, []),
    ("nb_kernel_launches", ctypes.c_uint64, []),
    ("nb_version", ctypes.c_char_p, []),
]

EXPORTED = [s[0] for s in _SIGS]


def lib():
    """Load libnbgpu.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(
                    f"{LIB} is missing: build it with paper_1905_13746_gb300.build() "
                    "(nvcc, sm_103a); there is no CPU fallback")
            handle = ctypes.CDLL(LIB)
            for name, res, args in _SIGS:
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def _check(status):
    if status != NB_OK:
        raise NbError(status, lib().nb_last_error().decode(errors="replace"))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- raw entry points (device pointers as ints) ---------------------------
def nb_fit(kind, X, dtype, n, F, ld, y, C, alpha=1.0, log_prior=None, var_smoothing=1e-9,
           aux=None, no_sync=False, stream=None):
    prior_buf = None
    if log_prior is not None:
        prior_buf = (ctypes.c_double * C)(*[float(v) for v in log_prior])
    opts = NbFitOpts(float(alpha), ctypes.cast(prior_buf, _P) if prior_buf else None,
                     float(var_smoothing), ctypes.pointer(aux) if aux else None, int(no_sync))
    out = _P()
    _check(lib().nb_fit(kind, X, dtype, n, F, ld, y, C, ctypes.byref(opts),
                        _stream_ptr(stream), ctypes.byref(out)))
    return out.value


def nb_refit(model, X, dtype, n, ld, y, alpha=1.0, log_prior=None, var_smoothing=1e-9,
             aux=None, no_sync=False, stream=None):
    prior_buf = None
    if log_prior is not None:
        prior_buf = (ctypes.c_double * len(log_prior))(*[float(v) for v in log_prior])
    opts = NbFitOpts(float(alpha), ctypes.cast(prior_buf, _P) if prior_buf else None,
                     float(var_smoothing), ctypes.pointer(aux) if aux else None, int(no_sync))
    _check(lib().nb_refit(model, X, dtype, n, ld, y, ctypes.byref(opts), _stream_ptr(stream)))


def nb_refit_gaussian_noalloc(model, X, n, ld, y, log_prior=None, var_smoothing=1e-9,
                              no_sync=False, stream=None):
    """Gaussian re-fit whose scratch is a fixed device array (no allocation)."""
    prior_buf = None
    if log_prior is not None:
        prior_buf = (ctypes.c_double * len(log_prior))(*[float(v) for v in log_prior])
    opts = NbFitOpts(1.0, ctypes.cast(prior_buf, _P) if prior_buf else None,
                     float(var_smoothing), None, int(no_sync))
    _check(lib().nb_refit_gaussian_noalloc(model, X, n, ld, y, ctypes.byref(opts),
                                           _stream_ptr(stream)))


def nb_kernel_launches():
    return int(lib().nb_kernel_launches())


def nb_score_group(model, X, dtype, n, ld, label, margin, logpost=None, want_logpost=False,
                   recheck=NB_RECHECK_LP, aux=None, stream=None, n_rechecked=None):
    opts = NbScoreOpts(int(want_logpost), int(recheck), ctypes.pointer(aux) if aux else None)
    _check(lib().nb_score_group(model, X, dtype, n, ld, label, margin, logpost,
                                ctypes.byref(opts), _stream_ptr(stream), n_rechecked))


def nb_model_free(model):
    if model:
        lib().nb_model_free(model)


def nb_last_error():
    return lib().nb_last_error().decode(errors="replace")


# ---- torch conveniences ----------------------------------------------------
def _torch_dtype_code(t, fp8=False):
    import torch
    m = {torch.float32: NB_F32, torch.uint8: NB_FP8E4M3 if fp8 else NB_U8,
         torch.bfloat16: NB_BF16, torch.float8_e4m3fn: NB_FP8E4M3}
    if hasattr(torch, "uint16"):
        m[torch.uint16] = NB_U16
    if t.dtype not in m:
        raise TypeError(f"unsupported feature dtype {t.dtype}")
    return m[t.dtype]


class Features:
    """A device feature matrix in one of the storage formats, plus side arrays."""

    def __init__(self, data, dtype_code=None, ovf_ptr=None, ovf_col=None, ovf_add=None,
                 row_exp=None):
        self.data = data
        self.dtype_code = _torch_dtype_code(data) if dtype_code is None else dtype_code
        self.ovf_ptr, self.ovf_col, self.ovf_add, self.row_exp = ovf_ptr, ovf_col, ovf_add, row_exp
        if data.dim() != 2 or (data.numel() > 0 and data.stride(1) != 1):
            raise ValueError("features must be a row-major matrix")

    @property
    def n(self):
        return self.data.shape[0]

    @property
    def F(self):
        return self.data.shape[1]

    @property
    def ld(self):
        return self.data.stride(0)

    def aux(self):
        if self.ovf_ptr is None and self.row_exp is None:
            return None
        p = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
        return NbAux(p(self.ovf_ptr), p(self.ovf_col), p(self.ovf_add), p(self.row_exp))

    def nbytes(self):
        b = self.data.numel() * self.data.element_size()
        for t in (self.ovf_ptr, self.ovf_col, self.ovf_add, self.row_exp):
            if t is not None:
                b += t.numel() * t.element_size()
        return b


def _labels(y, n):
    """Labels as the library reads them: n int32 values, contiguous."""
    import torch
    if not isinstance(y, torch.Tensor) or y.dtype != torch.int32 or y.dim() != 1 \
            or not y.is_contiguous() or y.shape[0] != n:
        raise TypeError("labels must be a contiguous 1-D int32 tensor of %d entries" % n)
    return y


def _sizes(s, n):
    """File sizes as the library reads them: n int64 values, contiguous."""
    import torch
    if not isinstance(s, torch.Tensor) or s.dtype != torch.int64 or s.dim() != 1 \
            or not s.is_contiguous() or s.shape[0] != n:
        raise TypeError("sizes must be a contiguous 1-D int64 tensor of %d entries" % n)
    return s


def as_features(X):
    return X if isinstance(X, Features) else Features(X)


class Model:
    """Owns an nb_model handle (freed with the object)."""

    def __init__(self, handle, kind, C, F):
        self.handle, self.kind, self.C, self.F = handle, kind, C, F

    def __del__(self):
        try:
            if self.handle:
                nb_model_free(self.handle)
        except Exception:
            pass
        self.handle = None

    def counts(self):
        import numpy as np
        c = np.zeros((self.C, self.F), np.uint64)
        nc = np.zeros(self.C, np.uint64)
        _check(lib().nb_model_counts(self.handle, c.ctypes.data, nc.ctypes.data))
        return c, nc

    def params(self):
        import numpy as np
        p0 = np.zeros((self.C, self.F), np.float64)
        p1 = np.zeros((self.C, self.F), np.float64) if self.kind == NB_GAUSSIAN else None
        lp = np.zeros(self.C, np.float64)
        _check(lib().nb_model_params(self.handle, p0.ctypes.data,
                                     p1.ctypes.data if p1 is not None else None, lp.ctypes.data))
        return p0, p1, lp

    def check(self):
        _check(lib().nb_model_check(self.handle))

    def tile_config(self):
        c = NbTileConfig()
        _check(lib().nb_get_tile_config(self.handle, ctypes.byref(c)))
        return (c.variant, c.stages, c.rows_per_stage, c.rows_per_warp)

    def set_tile_config(self, variant=NB_VARIANT_AUTO, stages=0, rows_per_stage=0,
                        rows_per_warp=0):
        c = NbTileConfig(variant, stages, rows_per_stage, rows_per_warp)
        _check(lib().nb_set_tile_config(self.handle, ctypes.byref(c)))

    def autotune(self, X, stream=None):
        """Time the scorer's candidate configurations on X; keep the fastest."""
        Xf = as_features(X)
        best = NbTileConfig()
        ms = ctypes.c_float(0)
        aux = Xf.aux()
        _check(lib().nb_autotune_score(self.handle, Xf.data.data_ptr(), Xf.dtype_code, Xf.n,
                                       Xf.ld, ctypes.byref(aux) if aux else None,
                                       _stream_ptr(stream), ctypes.byref(best),
                                       ctypes.byref(ms)))
        return (best.variant, best.stages, best.rows_per_stage, best.rows_per_warp), ms.value


def fit(X, y, C, kind=NB_MULTINOMIAL, alpha=1.0, log_prior=None, var_smoothing=1e-9,
        no_sync=False, stream=None):
    Xf = as_features(X)
    h = nb_fit(kind, Xf.data.data_ptr(), Xf.dtype_code, Xf.n, Xf.F, Xf.ld,
               _labels(y, Xf.n).data_ptr(), C,
               alpha=alpha, log_prior=log_prior, var_smoothing=var_smoothing, aux=Xf.aux(),
               no_sync=no_sync, stream=stream)
    return Model(h, kind, C, Xf.F)


def refit(model, X, y, alpha=1.0, log_prior=None, var_smoothing=1e-9, no_sync=False,
          stream=None):
    Xf = as_features(X)
    nb_refit(model.handle, Xf.data.data_ptr(), Xf.dtype_code, Xf.n, Xf.ld,
             _labels(y, Xf.n).data_ptr(),
             alpha=alpha, log_prior=log_prior, var_smoothing=var_smoothing, aux=Xf.aux(),
             no_sync=no_sync, stream=stream)
    return model


def score(model, X, want_logpost=True, recheck=NB_RECHECK_LP, stream=None, out=None):
    """Score a group; returns dict(label, margin, logpost, n_rechecked) of device tensors."""
    import torch
    Xf = as_features(X)
    dev = Xf.data.device
    n = Xf.n
    if out is None:
        out = {"label": torch.empty(n, dtype=torch.uint8, device=dev),
               "margin": torch.empty(n, dtype=torch.float32, device=dev),
               "logpost": torch.empty((n, model.C), dtype=torch.float32, device=dev)
               if want_logpost else None,
               "n_rechecked": torch.zeros(1, dtype=torch.int64, device=dev)}
    lp = out["logpost"].data_ptr() if want_logpost else None
    nb_score_group(model.handle, Xf.data.data_ptr(), Xf.dtype_code, n, Xf.ld,
                   out["label"].data_ptr(), out["margin"].data_ptr(), lp,
                   want_logpost=want_logpost, recheck=recheck, aux=Xf.aux(), stream=stream,
                   n_rechecked=out["n_rechecked"].data_ptr())
    return out


def score_path(model, X, recheck=NB_RECHECK_LP):
    """The NB_PATH_* scorer that score(model, X, recheck=recheck) launches."""
    Xf = as_features(X)
    r = lib().nb_score_path(model.handle, Xf.data.data_ptr(), Xf.dtype_code, Xf.ld, recheck)
    if r < 0:
        raise NbError(NB_EINVAL, nb_last_error())
    return r


# ---- batches of groups -----------------------------------------------------
class Batch:
    """Many groups (each with its own model slot and outputs) per launch.

    ``models``: Model objects (same F; two-class ones share one pipelined
    launch, many-class ones one general launch).  ``score(groups)`` takes a list
    of (slot, Features, out) where out is a dict of device tensors label,
    margin, logpost (as returned by ``outputs``).
    """

    def __init__(self, models, dtype_code, max_ld, max_groups, want_logpost=True,
                 recheck=NB_RECHECK_LP):
        self.models = list(models)
        arr = (_P * len(self.models))(*[m.handle for m in self.models])
        opts = NbScoreOpts(int(want_logpost), int(recheck), None)
        h = _P()
        _check(lib().nb_batch_create(arr, len(self.models), dtype_code, max_ld, max_groups,
                                     ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h.value
        self.want_logpost = want_logpost
        self._keep = []

    def __del__(self):
        try:
            if self.handle:
                lib().nb_batch_destroy(self.handle)
        except Exception:
            pass
        self.handle = None

    def outputs(self, slot, n, device="cuda"):
        import torch
        C = self.models[slot].C
        return {"label": torch.empty(n, dtype=torch.uint8, device=device),
                "margin": torch.empty(n, dtype=torch.float32, device=device),
                "logpost": torch.empty((n, C), dtype=torch.float32, device=device)
                if self.want_logpost else None}

    def score(self, groups, stream=None, n_rechecked=None):
        arr = (NbGroup * max(1, len(groups)))()
        for i, (slot, f, out) in enumerate(groups):
            aux = f.aux() or NbAux()
            arr[i] = NbGroup(slot, f.data.data_ptr(), f.n, f.ld, aux, out["label"].data_ptr(),
                             out["margin"].data_ptr(),
                             out["logpost"].data_ptr() if out.get("logpost") is not None else None)
        _check(lib().nb_batch_score(self.handle, arr, len(groups), _stream_ptr(stream),
                                    n_rechecked.data_ptr() if n_rechecked is not None else None))

    def capture(self, stream):
        _check(lib().nb_batch_capture(self.handle, _stream_ptr(stream)))


# ---- serving ----------------------------------------------------------------
class Server:
    """Continuous-batching server over resident models (see nb_server_create)."""

    def __init__(self, models, dtype_code, mem_budget=0, max_slots=64, want_logpost=True,
                 recheck=NB_RECHECK_LP):
        self.models = list(models)
        arr = (_P * len(self.models))(*[m.handle for m in self.models])
        opts = NbScoreOpts(int(want_logpost), int(recheck), None)
        h = _P()
        _check(lib().nb_server_create(arr, len(self.models), dtype_code, int(mem_budget),
                                      int(max_slots), ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h.value
        self.want_logpost = want_logpost
        self.F = self.models[0].F

    def close(self):
        if self.handle:
            lib().nb_server_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, model_id, n, device="cpu", pin=True):
        import torch
        C = self.models[model_id].C
        kw = {"device": device}
        mk = (lambda t: t.pin_memory()) if (device == "cpu" and pin) else (lambda t: t)
        return {"label": mk(torch.empty(n, dtype=torch.uint8, **kw)),
                "margin": mk(torch.empty(n, dtype=torch.float32, **kw)),
                "logpost": mk(torch.empty((n, C), dtype=torch.float32, **kw))
                if self.want_logpost else None}

    def submit(self, model_id, X, out):
        """X: (n x F) tensor on the host (pinned preferred) or the device."""
        t = ctypes.c_uint64(0)
        lp = out["logpost"].data_ptr() if out.get("logpost") is not None else None
        _check(lib().nb_classify_stream(self.handle, model_id, X.data_ptr(), X.shape[0],
                                        X.shape[1], out["label"].data_ptr(),
                                        out["margin"].data_ptr(), lp, ctypes.byref(t)))
        return t.value

    def submit_many(self, items, arrival_us=None):
        """items: list of (model_id, X, out) as for submit; arrival_us: optional
        list of scheduled arrival times on clock_us()'s clock.  Returns tickets."""
        k = len(items)
        if k == 0:
            return []
        mids = (ctypes.c_int * k)(*[m for m, _, _ in items])
        xs = (_P * k)(*[X.data_ptr() for _, X, _ in items])
        ns = (_i64 * k)(*[X.shape[0] for _, X, _ in items])
        for _, X, _ in items:
            if X.dim() != 2 or X.shape[1] != self.F:
                raise NbError(NB_EINVAL, "submit_many: every X must be (n x F)")
        lab = (_P * k)(*[o["label"].data_ptr() for _, _, o in items])
        mar = (_P * k)(*[o["margin"].data_ptr() for _, _, o in items])
        lps = (_P * k)(*[o["logpost"].data_ptr() if o.get("logpost") is not None else None
                         for _, _, o in items]) if self.want_logpost else None
        arr = (ctypes.c_double * k)(*arrival_us) if arrival_us is not None else None
        tk = (ctypes.c_uint64 * k)()
        done = ctypes.c_int(0)
        _check(lib().nb_classify_stream_batch(self.handle, k, mids, xs, ns, lab, mar, lps, arr,
                                              tk, ctypes.byref(done)))
        return list(tk)

    def submit_raw(self, model_ids, x_ptrs, n, label_ptrs, margin_ptrs, logpost_ptrs,
                   arrival_us=None):
        """Low-overhead burst submission from contiguous numpy arrays (int32
        model ids, uint64 pointers, int64 row counts, float64 arrival times);
        every pointer must address memory of the required size."""
        import numpy as np
        k = int(len(model_ids))
        if k == 0:
            return np.zeros(0, dtype=np.uint64)
        arrs = [np.ascontiguousarray(a, dtype=t) for a, t in
                ((model_ids, np.int32), (x_ptrs, np.uint64), (n, np.int64),
                 (label_ptrs, np.uint64), (margin_ptrs, np.uint64))]
        if any(len(a) != k for a in arrs):
            raise NbError(NB_EINVAL, "submit_raw: arrays of different lengths")
        lp = (np.ascontiguousarray(logpost_ptrs, dtype=np.uint64)
              if logpost_ptrs is not None else None)
        arr = (np.ascontiguousarray(arrival_us, dtype=np.float64)
               if arrival_us is not None else None)
        tk = np.zeros(k, dtype=np.uint64)
        done = ctypes.c_int(0)
        _check(lib().nb_classify_stream_batch(
            self.handle, k, *[a.ctypes.data for a in arrs[:3]], arrs[3].ctypes.data,
            arrs[4].ctypes.data, lp.ctypes.data if lp is not None else None,
            arr.ctypes.data if arr is not None else None, tk.ctypes.data, ctypes.byref(done)))
        return tk

    @staticmethod
    def clock_us():
        return lib().nb_clock_us()

    def wait(self, ticket, timeout_us=-1):
        _check(lib().nb_wait(self.handle, ticket, int(timeout_us)))

    def stats(self):
        a, b, c = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(lib().nb_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b),
                                     ctypes.byref(c)))
        return {"p50_us": a.value, "p99_us": b.value, "files_per_s": c.value}


# ---- packing ---------------------------------------------------------------
def pack_u8(X16, stream=None):
    """u16 counts (n x F) -> Features(u8 plane + overflow list)."""
    import torch
    n, F = X16.shape
    dev = X16.device
    ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    total = _i64(0)
    st = _stream_ptr(stream)
    _check(lib().nb_pack_u8_count(X16.data_ptr(), n, F, X16.stride(0), ptr.data_ptr(),
                                  ctypes.byref(total), st))
    ld_out = (F + 15) // 16 * 16
    plane = torch.empty((n, ld_out), dtype=torch.uint8, device=dev)[:, :F]
    col = torch.empty(max(total.value, 1), dtype=torch.int16, device=dev)
    add = torch.empty(max(total.value, 1), dtype=torch.int16, device=dev)
    _check(lib().nb_pack_u8_fill(X16.data_ptr(), n, F, X16.stride(0), plane.data_ptr(), ld_out,
                                 ptr.data_ptr(), col.data_ptr(), add.data_ptr(), st))
    return Features(plane, NB_U8, ptr, col, add)


def pack_bf16(X, stream=None):
    import torch
    n, F = X.shape
    src = NB_F32 if X.dtype == torch.float32 else NB_U16
    ld_out = (F + 7) // 8 * 8
    out = torch.empty((n, ld_out), dtype=torch.bfloat16, device=X.device)[:, :F]
    _check(lib().nb_pack_bf16(X.data_ptr(), src, n, F, X.stride(0), out.data_ptr(), ld_out,
                              _stream_ptr(stream)))
    return Features(out, NB_BF16)


def pack_fp8(X, stream=None):
    import torch
    n, F = X.shape
    src = NB_F32 if X.dtype == torch.float32 else NB_U16
    ld_out = (F + 15) // 16 * 16
    out = torch.empty((n, ld_out), dtype=torch.uint8, device=X.device)[:, :F]
    row_exp = torch.empty(n, dtype=torch.int8, device=X.device)
    _check(lib().nb_pack_fp8(X.data_ptr(), src, n, F, X.stride(0), out.data_ptr(), ld_out,
                             row_exp.data_ptr(), _stream_ptr(stream)))
    return Features(out, NB_FP8E4M3, row_exp=row_exp)


# ---- the group-wise method (Sec. 3 size groups and top-k opcodes, Sec. 4
# per-group models and the small-group rule) ------------------------------------
BIN_BYTES, N_BINS, MIN_FILES = 5 * 1024, 100, 6


def group_fallback(class_counts, min_files=MIN_FILES):
    """Host: model group of every size group from (n_bins x C) training-file
    counts (nb_group_fallback)."""
    import numpy as np
    cc = np.ascontiguousarray(class_counts, dtype=np.int64)
    n_bins, C = cc.shape
    out = np.zeros(n_bins, np.int32)
    _check(lib().nb_group_fallback(cc.ctypes.data, n_bins, C, int(min_files), out.ctypes.data))
    return out


def route(sizes, bin_bytes=BIN_BYTES, n_bins=N_BINS, model_of=None, n_groups=None, y=None,
          C=2, want_order=True, stream=None):
    """Route files by size (nb_route).  sizes: device int64 tensor.  Returns
    dict(group, order, offsets, class_counts (with y), status) of device tensors."""
    import torch
    dev = sizes.device
    n = sizes.shape[0]
    _sizes(sizes, n)
    if y is not None:
        _labels(y, n)
    G = int(n_groups) if n_groups is not None else n_bins
    ws = int(lib().nb_route_workspace(n, G))
    work = torch.empty(max(ws, 8), dtype=torch.uint8, device=dev)
    group = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    order = torch.empty(max(n, 1), dtype=torch.int64, device=dev) if want_order else None
    offsets = torch.empty(G + 1, dtype=torch.int64, device=dev)
    cc = torch.empty((n_bins, C), dtype=torch.int64, device=dev) if y is not None else None
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    mo = None
    if model_of is not None:
        mo = torch.as_tensor(model_of, dtype=torch.int32).to(dev)
    _check(lib().nb_route(sizes.data_ptr(), n, int(bin_bytes), int(n_bins),
                          mo.data_ptr() if mo is not None else None, G,
                          y.data_ptr() if y is not None else None, int(C), group.data_ptr(),
                          order.data_ptr() if order is not None else None, offsets.data_ptr(),
                          cc.data_ptr() if cc is not None else None, work.data_ptr(), ws,
                          status.data_ptr(), _stream_ptr(stream)))
    return {"group": group[:n], "order": order[:n] if order is not None else None,
            "offsets": offsets, "class_counts": cc, "status": status, "_keep": (work, mo)}


def select_features(models, k, norm=NB_SELECT_TOTAL, stream=None):
    """Top-k opcodes of two-class models (nb_select_features): int32 (n x k)."""
    import torch
    arr = (_P * len(models))(*[m.handle for m in models])
    cols = torch.empty((len(models), k), dtype=torch.int32, device="cuda")
    _check(lib().nb_select_features(arr, len(models), int(k), int(norm), cols.data_ptr(),
                                    _stream_ptr(stream)))
    return cols


def padded_ld(k, dtype_code):
    """Row pitch (elements) of gathered rows: 16-byte aligned."""
    es = 1 if dtype_code == NB_U8 else 4
    return (k * es + 15) // 16 * 16 // es


def gather(X, cols=None, k=None, order=None, group=None, n_groups=None, n=None, ld_out=None,
           stream=None, status=None):
    """nb_gather: rows of X (U8 or F32 tensor) by ``order``, columns by each
    row's group's row of ``cols`` (int32 device tensor n_groups x k)."""
    import torch
    dt = _torch_dtype_code(X)
    F = X.shape[1]
    if k is None:
        k = cols.shape[-1] if cols is not None else F
    if n is None:
        n = order.shape[0] if order is not None else X.shape[0]
    if ld_out is None:
        ld_out = padded_ld(k, dt)
    out = torch.empty((n, ld_out), dtype=X.dtype, device=X.device)
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=X.device)
    G = int(n_groups) if n_groups is not None else (cols.shape[0] if cols is not None and
                                                     cols.dim() == 2 else 1)
    _check(lib().nb_gather(X.data_ptr(), dt, X.stride(0), F, X.shape[0], n,
                           order.data_ptr() if order is not None else None,
                           group.data_ptr() if group is not None else None, G,
                           cols.data_ptr() if cols is not None else None, int(k),
                           out.data_ptr(), ld_out, st.data_ptr(), _stream_ptr(stream)))
    return out[:, :k], st


class Groupwise:
    """Group-wise classifier over full opcode histograms (nb_groupwise_*)."""

    def __init__(self, models, cols, model_of, F_full, dtype_code=NB_U8, max_files=1 << 20,
                 bin_bytes=BIN_BYTES, want_logpost=True, recheck=NB_RECHECK_LP):
        import numpy as np
        self.models = list(models)
        self.k = self.models[0].F
        arr = (_P * len(self.models))(*[m.handle for m in self.models])
        mo = np.ascontiguousarray(model_of, dtype=np.int32)
        self.cols = cols.contiguous()
        opts = NbScoreOpts(int(want_logpost), int(recheck), None)
        h = _P()
        _check(lib().nb_groupwise_create(arr, len(self.models), self.cols.data_ptr(), self.k,
                                          mo.ctypes.data, mo.shape[0], int(bin_bytes),
                                          int(F_full), dtype_code, int(max_files),
                                          ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h.value
        self.want_logpost = want_logpost

    def close(self):
        if self.handle:
            lib().nb_groupwise_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def classify(self, X, sizes, stream=None, out=None):
        """X: (n x F_full) device histograms, sizes: device int64 (n).  Returns
        dict(label, margin, logpost, n_rechecked) in the files' order."""
        import torch
        n, dev = X.shape[0], X.device
        if out is None:
            out = {"label": torch.empty(n, dtype=torch.uint8, device=dev),
                   "margin": torch.empty(n, dtype=torch.float32, device=dev),
                   "logpost": torch.empty((n, 2), dtype=torch.float32, device=dev)
                   if self.want_logpost else None,
                   "n_rechecked": torch.zeros(1, dtype=torch.int64, device=dev)}
        lp = out["logpost"].data_ptr() if out.get("logpost") is not None else None
        _check(lib().nb_groupwise_classify(self.handle, X.data_ptr(), X.stride(0),
                                           sizes.data_ptr(), n, out["label"].data_ptr(),
                                           out["margin"].data_ptr(), lp, _stream_ptr(stream),
                                           out["n_rechecked"].data_ptr()))
        return out

    def status(self):
        v = ctypes.c_int(0)
        _check(lib().nb_groupwise_status(self.handle, ctypes.byref(v)))
        return v.value


def fit_groupwise(X, y, sizes, k, norm=NB_SELECT_TOTAL, alpha=1.0, bin_bytes=BIN_BYTES,
                  n_bins=N_BINS, min_files=MIN_FILES, stream=None):
    """Train the per-group models of the method on the device.

    X: (n x F) U8 or F32 full histograms, y: int32 labels, sizes: int64 file
    sizes (all device tensors).  Routes the files (labels counted per size
    group), applies the small-group rule, fits each trained group on all
    opcodes, ranks its opcodes, and fits it again on its top k.  Returns
    dict(models, cols, model_of (slot per size group), groups (size group of
    each slot), full_models)."""
    import torch
    n, F = X.shape
    r = route(sizes, bin_bytes, n_bins, y=y, C=2, stream=stream)
    cc = r["class_counts"].cpu().numpy()
    mo_bins = group_fallback(cc, min_files)
    trained = sorted(set(mo_bins.tolist()))
    slot = {g: i for i, g in enumerate(trained)}
    offs = r["offsets"].cpu().tolist()
    order = r["order"]
    Xs, _ = gather(X, order=order, stream=stream)          # rows sorted by size group
    # labels follow their rows (a 4-byte gather of one column)
    ys = gather(y.view(torch.float32).reshape(n, 1), order=order, ld_out=1,
                stream=stream)[0].reshape(n).view(torch.int32)
    full = []
    for g in trained:
        a, b = offs[g], offs[g + 1]
        full.append(fit(Xs[a:b], ys[a:b], 2, alpha=alpha, stream=stream))
    cols = select_features(full, k, norm, stream=stream)
    models = []
    for i, g in enumerate(trained):
        a, b = offs[g], offs[g + 1]
        Xg, _ = gather(Xs[a:b], cols[i:i + 1], stream=stream)
        models.append(fit(Xg, ys[a:b], 2, alpha=alpha, stream=stream))
    model_of = [slot[int(m)] for m in mo_bins]
    return {"models": models, "cols": cols, "model_of": model_of, "groups": trained,
            "full_models": full, "class_counts": cc}
