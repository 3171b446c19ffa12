"""The allocation-free Gaussian re-fit against the ordinary one.

nb_refit_gaussian_noalloc exists for callers that may not allocate device
memory when they re-train (a fixed memory budget, a CUDA graph already
instantiated, a runtime that forbids allocation after start-up); it keeps its
partial sums in a fixed device array of the library instead of
cudaMallocAsync scratch.  Its results must equal nb_refit's, call after call,
whether this file runs alone in a fresh process or after the other tests.
The file name makes pytest collect it last.
"""
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


def test_noalloc_refit_matches_refit_twice():
    assert torch.cuda.is_available()
    nb.build()
    w = synth.gaussian_workload(synth.seed_for(1))
    X0 = torch.from_numpy(w["X_fit"]).cuda()
    y0 = torch.from_numpy(w["y_fit"]).cuda()
    ref = nb.fit(X0, y0, 2, kind=nb.NB_GAUSSIAN, log_prior=w["log_prior"])
    new = nb.fit(X0, y0, 2, kind=nb.NB_GAUSSIAN, log_prior=w["log_prior"])
    Xs = torch.from_numpy(w["X_score"]).cuda()
    for call, (seed, n_per) in enumerate([(11, 1500), (12, 3001)]):
        X, y = _data(seed, n_per, w["X_fit"].shape[1])
        nb.refit(ref, X, y, log_prior=w["log_prior"])
        nb.nb_refit_gaussian_noalloc(new.handle, X.data_ptr(), X.shape[0], X.stride(0),
                                     y.data_ptr(), log_prior=w["log_prior"])
        torch.cuda.synchronize()
        mu_r, var_r, lp_r = ref.params()
        mu_n, var_n, lp_n = new.params()
        assert np.allclose(mu_n, mu_r, rtol=1e-12, atol=1e-12), call
        assert np.allclose(var_n, var_r, rtol=1e-12, atol=0), call
        assert (lp_n == lp_r).all(), call
        r = nb.score(ref, Xs)
        s = nb.score(new, Xs)
        assert torch.equal(r["label"], s["label"]), call
        lr, ls = r["logpost"].cpu().numpy(), s["logpost"].cpu().numpy()
        assert (np.abs(ls - lr) <= 1e-5 * np.maximum(1.0, np.abs(lr))).all(), call


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
