"""The many-class Gaussian tensor-core scorer (tcgen05, 3 <= C <= 64 classes,
F <= 8192 FP32 features) against the FP64 oracle.  Its FP32 accumulation of
FP16 limb products is not exact; a rigorous per-row bound sends the rows it does
not settle to the FP64 recheck, so labels are exact after the recheck in the
label mode, and log posteriors meet the usual tolerance when the tensor-core
scorer is forced in the log-posterior mode (Sec. 4 posterior and decision
rule, class-conditional Gaussians)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests._common import compare, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    nb.build()
    nb.lib()


def _data(seed, C, F, n_fit_per_class, n_score, spread=10.0):
    """Class means U(0, spread), deviations U(0.5, 3), x ~ N(mu_y, sd_y^2):
    the real-feature generator at C classes and F features."""
    w = synth.gaussian_workload(seed, F=F, C=C, n_fit_per_class=n_fit_per_class,
                                n_score_per_class=(n_score + C - 1) // C, spread=spread)
    return w["X_fit"], w["y_fit"], w["X_score"][:n_score]


def _fit(X, y, C):
    return nb.fit(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), C,
                  kind=nb.NB_GAUSSIAN)


def _rows(Xs):
    """Device rows with a pitch of a multiple of 16 bytes (the tensor map's
    stride rule), as a view of the first F columns."""
    n, F = Xs.shape
    ld = (F + 3) // 4 * 4
    buf = torch.full((n, ld), 7.0, dtype=torch.float32, device="cuda")
    buf[:, :F] = torch.from_numpy(Xs).cuda()
    return buf[:, :F]


def _score(model, Xs, recheck, want_lp=True):
    X = _rows(Xs)
    return X, to_np(nb.score(model, X, want_logpost=want_lp, recheck=recheck))


# (classes, features, files scored): one feature, one partial and one full
# 8-feature stage, partial and full 32-feature row boxes, several 128-file
# tiles with ragged tails, the 64-class shape up to the largest F
CASES = [(3, 1, 5), (3, 7, 300), (5, 8, 129), (16, 33, 1000), (17, 200, 2000),
         (33, 64, 3001), (64, 64, 2560), (64, 1024, 1500), (64, 8192, 300)]


@pytest.mark.parametrize("C,F,n", CASES)
def test_gaussian_tensor_scorer_labels_exact(C, F, n):
    Xf, yf, Xs = _data(1200 + C + F, C, F, 20, n)
    model = _fit(Xf, yf, C)
    X, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    assert nb.score_path(model, X, nb.NB_RECHECK_LABEL) == nb.NB_PATH_TENSOR_GAUSS
    ref = oracle.score(Xs, oracle.gauss_fit(Xf, yf, C))
    compare(res, ref, check_lp=False)
    # unrechecked rows: the FP32 scores are within the bound, far below 1e-3
    # relative on these margins
    mar = res["margin"].astype(np.float64)
    assert (np.abs(mar - ref["margin"]) <= 1e-3 * np.maximum(1.0, np.abs(ref["margin"]))).all()


@pytest.mark.parametrize("C,F,n", [(3, 7, 300), (16, 33, 1000), (64, 1024, 700)])
def test_gaussian_tensor_scorer_forced_log_posterior(C, F, n):
    # the tensor-core scorer in the log-posterior mode: rows whose bound is
    # above the tolerance go to FP64, so every output meets it
    Xf, yf, Xs = _data(1300 + C + F, C, F, 20, n)
    model = _fit(Xf, yf, C)
    model.set_tile_config(nb.NB_VARIANT_PIPELINED, 0, 0, 0)
    X, res = _score(model, Xs, nb.NB_RECHECK_LP)
    assert nb.score_path(model, X, nb.NB_RECHECK_LP) == nb.NB_PATH_TENSOR_GAUSS
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)))


def test_gaussian_default_log_posterior_mode_uses_cuda_cores():
    Xf, yf, Xs = _data(1400, 8, 40, 20, 500)
    model = _fit(Xf, yf, 8)
    X, res = _score(model, Xs, nb.NB_RECHECK_LP)
    assert nb.score_path(model, X, nb.NB_RECHECK_LP) == nb.NB_PATH_GENERAL
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, 8)))


@pytest.mark.parametrize("C,F", [(16, 256), (64, 1024)])
def test_gaussian_close_classes_go_to_fp64(C, F):
    # every class drawn from one distribution: the fitted classes differ by
    # sampling noise alone, margins are of the order of the bound, a share of
    # the rows goes to FP64, and every label still matches
    rng = np.random.default_rng(1500 + C)
    mu = rng.uniform(0.0, 10.0, size=F)
    sd = rng.uniform(0.5, 3.0, size=F)
    yf = np.concatenate([np.arange(C), rng.integers(0, C, 30 * C - C)]).astype(np.int32)
    Xf = rng.normal(mu, sd, size=(yf.shape[0], F)).astype(np.float32)
    Xs = rng.normal(mu, sd, size=(2000, F)).astype(np.float32)
    model = _fit(Xf, yf, C)
    _, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)), check_lp=False)
    assert res["n_rechecked"] > 0


def test_gaussian_tensor_and_cuda_core_scorers_agree():
    C, F = 48, 300
    Xf, yf, Xs = _data(1600, C, F, 20, 4000)
    model = _fit(Xf, yf, C)
    X = _rows(Xs)
    tc = to_np(nb.score(model, X, recheck=nb.NB_RECHECK_LABEL))
    model.set_tile_config(nb.NB_VARIANT_REGISTER, 0, 0, 0)
    assert nb.score_path(model, X, nb.NB_RECHECK_LABEL) == nb.NB_PATH_GENERAL
    cc = to_np(nb.score(model, X, recheck=nb.NB_RECHECK_LABEL))
    assert (tc["label"] == cc["label"]).all()
    d = np.abs(tc["lp"].astype(np.float64) - cc["lp"]) / np.maximum(1.0, np.abs(cc["lp"]))
    assert d.max() < 1e-3


def test_gaussian_tensor_scorer_out_of_range_rows():
    # a feature value whose centred square leaves the FP16 range marks its row
    # for FP64; NaN rows likewise; the rest are untouched
    C, F = 10, 96
    Xf, yf, Xs = _data(1700, C, F, 20, 600)
    Xs = Xs.copy()
    Xs[3, 5] = 1e6
    Xs[200, 95] = -3e4
    Xs[301, 0] = 400.0
    model = _fit(Xf, yf, C)
    _, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    ref = oracle.score(Xs, oracle.gauss_fit(Xf, yf, C))
    compare(res, ref, check_lp=False)
    assert res["n_rechecked"] >= 3


def test_gaussian_tensor_scorer_unaligned_falls_back():
    C, F = 6, 30
    Xf, yf, Xs = _data(1800, C, F, 20, 300)
    model = _fit(Xf, yf, C)
    big = torch.zeros((Xs.shape[0], F + 3), dtype=torch.float32, device="cuda")
    big[:, 1:F + 1] = torch.from_numpy(Xs).cuda()
    X = big[:, 1:F + 1]   # 4-byte offset, ld = F + 3
    assert nb.score_path(model, X, nb.NB_RECHECK_LABEL) == nb.NB_PATH_GENERAL
    res = to_np(nb.score(model, X, recheck=nb.NB_RECHECK_LABEL))
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)), check_lp=False)


@pytest.mark.parametrize("C", [33, 64])
def test_gaussian_fit_many_classes(C):
    # the fit's narrower feature tile above 32 classes: FP64 moments within
    # 1e-12 of the oracle's
    Xf, yf, _ = _data(1900 + C, C, 150, 25, 1)
    model = _fit(Xf, yf, C)
    ref = oracle.gauss_fit(Xf, yf, C)
    mu, var, lpi = model.params()
    assert np.allclose(mu, ref["mu"], rtol=1e-12, atol=1e-12)
    assert np.allclose(var, ref["var"], rtol=1e-12, atol=0)
    assert np.allclose(lpi, ref["log_pi"], rtol=0, atol=1e-14)


def test_gaussian_refit_rebuilds_tensor_tables():
    # refit (and the allocation-free refit) rederive the tensor-core tables
    C, F = 20, 120
    Xa, ya, Xs = _data(2000, C, F, 20, 800)
    Xb, yb, _ = _data(2001, C, F, 20, 1)
    model = _fit(Xa, ya, C)
    nb.refit(model, torch.from_numpy(Xb).cuda(), torch.from_numpy(yb).cuda())
    _, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xb, yb, C)), check_lp=False)
    # the allocation-free refit on new rows rederives them too
    Xc, yc, _ = _data(2002, C, F, 20, 1)
    Xd = torch.from_numpy(Xc).cuda()
    yd = torch.from_numpy(yc).cuda()
    nb.nb_refit_gaussian_noalloc(model.handle, Xd.data_ptr(), Xd.shape[0], Xd.stride(0),
                                 yd.data_ptr())
    _, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xc, yc, C)), check_lp=False)


@pytest.mark.parametrize("C,F", [(64, 64), (64, 1024), (16, 256)])
def test_gaussian_log_posterior_mode_rechecks_few_rows(C, F):
    # the CUDA-core scorer's log-posterior test weighs each class's bound
    # against that class's own distance from the top: on separated classes
    # almost no row needs FP64, and the results meet the tolerance
    Xf, yf, Xs = _data(1600 + C + F, C, F, 40, 3000)
    model = _fit(Xf, yf, C)
    X, res = _score(model, Xs, nb.NB_RECHECK_LP)
    assert nb.score_path(model, X, nb.NB_RECHECK_LP) == nb.NB_PATH_GENERAL
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)))
    assert res["n_rechecked"] <= 30, res["n_rechecked"]


def test_gaussian_log_posterior_mode_close_classes():
    # classes that differ by sampling noise alone: many rows go to FP64 in the
    # log-posterior mode, and every label and log posterior still matches
    C, F = 16, 128
    rng = np.random.default_rng(1700)
    mu = rng.uniform(0.0, 10.0, size=F)
    sd = rng.uniform(0.5, 3.0, size=F)
    yf = np.concatenate([np.arange(C), rng.integers(0, C, 30 * C - C)]).astype(np.int32)
    Xf = rng.normal(mu, sd, size=(yf.shape[0], F)).astype(np.float32)
    Xs = rng.normal(mu, sd, size=(2000, F)).astype(np.float32)
    model = _fit(Xf, yf, C)
    _, res = _score(model, Xs, nb.NB_RECHECK_LP)
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)))
    assert res["n_rechecked"] > 0


def test_gaussian_tensor_scorer_empty_and_single_row():
    Xf, yf, Xs = _data(1800, 6, 40, 20, 200)
    model = _fit(Xf, yf, 6)
    X0, r0 = _score(model, Xs[:0], nb.NB_RECHECK_LABEL)
    assert r0["label"].size == 0
    for n in (1, 129):
        X, res = _score(model, Xs[:n], nb.NB_RECHECK_LABEL)
        assert nb.score_path(model, X, nb.NB_RECHECK_LABEL) == nb.NB_PATH_TENSOR_GAUSS
        compare(res, oracle.score(Xs[:n], oracle.gauss_fit(Xf, yf, 6)), check_lp=False)


# the CUDA-core Gaussian scorer's shapes: 4- and 16-class blocks, groups of 8,
# 16 and 32 lanes per row (F up to 128, 512 and beyond), staged feature chunks
# with a ragged last one, block tiles with a ragged last one; the 64-class case
# past the tensor-core scorer's largest F
GEN_CASES = [(2, 7, 301), (3, 100, 517), (4, 300, 1000), (5, 33, 259), (17, 200, 700),
             (64, 64, 1029), (48, 600, 333), (64, 9000, 70)]


@pytest.mark.parametrize("C,F,n", GEN_CASES)
@pytest.mark.parametrize("rc", ["label", "lp"])
def test_gaussian_cuda_core_scorer_shapes(C, F, n, rc):
    mode = nb.NB_RECHECK_LP if rc == "lp" else nb.NB_RECHECK_LABEL
    Xf, yf, Xs = _data(1900 + C + F, C, F, 20, n)
    model = _fit(Xf, yf, C)
    model.set_tile_config(nb.NB_VARIANT_REGISTER, 0, 0, 0)
    X, res = _score(model, Xs, mode)
    assert nb.score_path(model, X, mode) == nb.NB_PATH_GENERAL
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)), check_lp=rc == "lp")


def test_gaussian_cuda_core_scorer_close_classes_label_mode():
    # classes that differ by sampling noise: the bound, not the margin,
    # decides; the rows it does not settle go to FP64 and every label matches
    C, F = 24, 300
    rng = np.random.default_rng(1950)
    mu = rng.uniform(0.0, 10.0, size=F)
    sd = rng.uniform(0.5, 3.0, size=F)
    yf = np.concatenate([np.arange(C), rng.integers(0, C, 30 * C - C)]).astype(np.int32)
    Xf = rng.normal(mu, sd, size=(yf.shape[0], F)).astype(np.float32)
    Xs = rng.normal(mu, sd, size=(1500, F)).astype(np.float32)
    model = _fit(Xf, yf, C)
    model.set_tile_config(nb.NB_VARIANT_REGISTER, 0, 0, 0)
    _, res = _score(model, Xs, nb.NB_RECHECK_LABEL)
    compare(res, oracle.score(Xs, oracle.gauss_fit(Xf, yf, C)), check_lp=False)
