"""The allocation-free Gaussian re-fit against the ordinary one.

nb_refit_gaussian_noalloc exists for callers that may not allocate device
memory when they re-train (a fixed memory budget, a CUDA graph already
instantiated, a runtime that forbids allocation after start-up); it keeps its
partial sums in a fixed device array of the library instead of
cudaMallocAsync scratch.  Its results must be the same bits as nb_refit's,
call after call, at sizes on both sides of the row-chunk switch (65,536 rows),
and a call must not allocate device memory, whether this file runs alone in a
fresh process or after the other tests.  The file name makes pytest collect it
last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")


def _data(seed, n_per, F, C=2):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0, 10, size=(C, F))
    sd = rng.uniform(0.5, 3, size=(C, F))
    y = np.repeat(np.arange(C, dtype=np.int32), n_per)
    y = y[rng.permutation(y.shape[0])]
    X = rng.normal(mu[y], sd[y]).astype(np.float32)
    return torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()


def _cudart():
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13",
                 "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.fail("the CUDA runtime library could not be loaded")


class _DefaultPool:
    """High-water mark of the device's default stream-ordered memory pool
    (the pool nb_refit's cudaMallocAsync scratch comes from)."""
    USED_CURRENT, USED_HIGH = 7, 8   # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh

    def __init__(self):
        self.rt = _cudart()
        self.pool = ctypes.c_void_p()
        dev = torch.cuda.current_device()
        assert self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_HIGH, ctypes.byref(zero)) == 0

    def used(self):
        return self._get(self.USED_CURRENT)

    def high(self):
        return self._get(self.USED_HIGH)


def test_noalloc_refit_matches_refit_twice():
    assert torch.cuda.is_available()
    nb.build()
    w = synth.gaussian_workload(synth.seed_for(1))
    F = w["X_fit"].shape[1]
    X0 = torch.from_numpy(w["X_fit"]).cuda()
    y0 = torch.from_numpy(w["y_fit"]).cuda()
    ref = nb.fit(X0, y0, 2, kind=nb.NB_GAUSSIAN, log_prior=w["log_prior"])
    new = nb.fit(X0, y0, 2, kind=nb.NB_GAUSSIAN, log_prior=w["log_prior"])
    Xs = torch.from_numpy(w["X_score"]).cuda()
    # 32-row partial sums below 65,536 rows, 256-row ones above: both sides
    for call, (seed, n_per) in enumerate([(11, 1500), (12, 35_001), (14, 3001)]):
        X, y = _data(seed, n_per, F)
        prior = w["log_prior"] if call != 1 else None
        nb.refit(ref, X, y, log_prior=prior)
        nb.nb_refit_gaussian_noalloc(new.handle, X.data_ptr(), X.shape[0], X.stride(0),
                                     y.data_ptr(), log_prior=prior)
        torch.cuda.synchronize()
        mu_r, var_r, lp_r = ref.params()
        mu_n, var_n, lp_n = new.params()
        assert np.array_equal(mu_n, mu_r), call
        assert np.array_equal(var_n, var_r), call
        assert np.array_equal(lp_n, lp_r), call
        r = nb.score(ref, Xs)
        s = nb.score(new, Xs)
        assert torch.equal(r["label"], s["label"]), call
        assert torch.equal(r["margin"], s["margin"]), call
        assert torch.equal(r["logpost"], s["logpost"]), call


def test_noalloc_allocates_nothing():
    w = synth.gaussian_workload(synth.seed_for(1))
    F = w["X_fit"].shape[1]
    model = nb.fit(torch.from_numpy(w["X_fit"]).cuda(), torch.from_numpy(w["y_fit"]).cuda(), 2,
                   kind=nb.NB_GAUSSIAN)
    X, y = _data(15, 40_000, F)
    pool = _DefaultPool()

    def call():
        nb.nb_refit_gaussian_noalloc(model.handle, X.data_ptr(), X.shape[0], X.stride(0),
                                     y.data_ptr())
        torch.cuda.synchronize()

    call()
    free0 = torch.cuda.mem_get_info()[0]
    torch_alloc0 = torch.cuda.memory_allocated()
    used0 = pool.used()
    pool.reset_high()
    call()
    call()
    assert pool.high() == used0, "the call took memory from the default stream-ordered pool"
    assert torch.cuda.mem_get_info()[0] == free0, "device memory was allocated"
    assert torch.cuda.memory_allocated() == torch_alloc0
    # the ordinary re-fit, for contrast, does draw its scratch from that pool
    pool.reset_high()
    nb.refit(model, X, y)
    torch.cuda.synchronize()
    assert pool.high() > used0


def test_noalloc_rejects_requests_beyond_its_scratch():
    Xs, ys = _data(13, 500, 256)
    model = nb.fit(Xs, ys, 2, kind=nb.NB_GAUSSIAN)
    # ceil(400000 / 256) * (2 + 1) * 256 + 2 * 256 = 1,200,896 doubles > 2^20
    X = torch.zeros((400_000, 256), dtype=torch.float32, device="cuda")
    y = torch.zeros(400_000, dtype=torch.int32, device="cuda")
    with pytest.raises(nb.NbError) as ei:
        nb.nb_refit_gaussian_noalloc(model.handle, X.data_ptr(), X.shape[0], X.stride(0),
                                     y.data_ptr())
    assert ei.value.status == nb.NB_EINVAL
    assert "scratch" in str(ei.value)
