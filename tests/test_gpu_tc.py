"""The many-class tensor-core scorer (tcgen05, 3 <= C <= 64 classes, u8
storage with or without the overflow list, BF16 and FP8 E4M3 rows, row pitch a
multiple of 16 bytes) against the
FP64 oracle, element by element, and against the CUDA-core scorer of the same
model.  Its fixed-point weights make the FP32 accumulation exact, so the
rigorous error bound stays small and the FP64 recheck rare even in the
log-posterior mode (Sec. 4 posterior and decision rule)."""
import numpy as np
import pytest
import torch

from tests._common import compare, count_matrix, oracle_mn, stored, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    nb.build()
    nb.lib()


def _model(fmt, X, y, C):
    f, v = stored(X, fmt)
    return nb.fit(f, torch.from_numpy(y).cuda(), C), v


# (classes, features, files scored): one to several 128-file tiles with ragged
# tails, a single 64-feature stage, partial 64- and 256-feature stages, and the
# 64-class / 8192-feature shape of the many-class workload
CASES = [(3, 64, 1), (3, 528, 777), (5, 1000, 300), (16, 2048, 3001), (17, 1024, 129),
         (33, 1040, 1000), (64, 4096, 2560), (64, 8192, 1500)]


@pytest.mark.parametrize("C,F,n", CASES)
def test_tensor_scorer_matches_oracle(C, F, n):
    X, y, _ = count_matrix(900 + C + F, 2500 + n, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X[:2500], y[:2500], C)
    fsc, vsc = stored(X[2500:], "u8")
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    _, ref = oracle_mn(vfit, y[:2500], C, vsc)
    compare(res, ref)
    # exact accumulation: only the weight quantisation bound remains
    assert res["n_rechecked"] <= max(3, n // 100), res["n_rechecked"]


@pytest.mark.parametrize("C,F", [(16, 1024), (5, 256)])
def test_tensor_scorer_with_overflow_list(C, F):
    X, y, _ = count_matrix(950 + C, 4000, F, C=C, conc=0.1, clip=65535)
    assert (X > 255).any()
    model, vfit = _model("u8ovf", X[:2000], y[:2000], C)
    fsc, vsc = stored(X[2000:], "u8ovf")
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    _, ref = oracle_mn(vfit, y[:2000], C, vsc)
    compare(res, ref)


@pytest.mark.parametrize("C,F", [(16, 512), (64, 1024)])
def test_tensor_and_cuda_core_scorers_agree(C, F):
    X, y, _ = count_matrix(970 + C, 5000, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X[:2000], y[:2000], C)
    fsc, vsc = stored(X[2000:], "u8")
    tc = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LABEL))
    model.set_tile_config(nb.NB_VARIANT_REGISTER, 0, 0, 0)   # CUDA-core scorer
    cc = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LABEL))
    model.set_tile_config(nb.NB_VARIANT_AUTO, 0, 0, 0)
    assert (tc["label"] == cc["label"]).all()
    d = np.abs(tc["lp"].astype(np.float64) - cc["lp"]) / np.maximum(1.0, np.abs(cc["lp"]))
    assert d.max() < 1e-4
    _, ref = oracle_mn(vfit, y[:2000], C, vsc)
    compare(tc, ref, check_lp=False)


def test_tensor_scorer_zero_rows_and_ties():
    # all-zero rows score the log priors alone; identical class profiles tie
    C, F = 4, 256
    X, y, _ = count_matrix(990, 3000, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X, y, C)
    Z = np.zeros((300, F), np.uint8)
    Z[::3] = X[:100]
    fsc, vsc = stored(Z, "u8")
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    _, ref = oracle_mn(vfit, y, C, vsc)
    compare(res, ref)


def test_tensor_scorer_heavy_rows_redone_exactly():
    # rows with 2^17 or more stored counts leave the single-accumulation pass
    # and are scored again with exact 512-feature chunks
    C, F = 8, 1024
    X, y, _ = count_matrix(995, 6000, F, C=C, conc=0.1, clip=255)
    rng = np.random.default_rng(7)
    heavy = rng.choice(np.arange(3000, 6000), 400, replace=False)
    X[heavy] = rng.integers(150, 256, size=(400, F))        # >= 153,600 counts
    model, vfit = _model("u8", X[:3000], y[:3000], C)
    fsc, vsc = stored(X[3000:], "u8")
    _, ref = oracle_mn(vfit, y[:3000], C, vsc)
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    compare(res, ref)
    lab = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LABEL))
    compare(lab, ref, check_lp=False)
    assert lab["n_rechecked"] <= 30, lab["n_rechecked"]


# BF16 and FP8 E4M3 rows: counts up to 255 are exact in BF16; E4M3 rounds them
# (row scale 2^0), and the oracle scores the stored values
@pytest.mark.parametrize("fmt", ["bf16", "fp8"])
@pytest.mark.parametrize("C,F,n", [(5, 1000, 777), (17, 520, 129), (64, 4096, 1300)])
def test_tensor_scorer_bf16_fp8_rows(fmt, C, F, n):
    X, y, _ = count_matrix(1100 + C + F, 2500 + n, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X[:2500], y[:2500], C)
    fsc, vsc = stored(X[2500:], fmt)
    assert nb.score_path(model, fsc) == nb.NB_PATH_TENSOR
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    _, ref = oracle_mn(vfit, y[:2500], C, vsc)
    compare(res, ref)
    assert res["n_rechecked"] <= max(3, n // 100), res["n_rechecked"]
    lab = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LABEL))
    compare(lab, ref, check_lp=False)


def test_tensor_scorer_fp8_row_scales():
    # rows whose largest count exceeds 448 carry a row scale 2^e: e = 1 stays on
    # the tensor cores (scores scaled in the epilogue), e >= 2 goes to FP64
    C, F = 8, 512
    X, y, _ = count_matrix(1150, 5000, F, C=C, conc=0.1, clip=3000)
    model, vfit = _model("u16", X[:2500], y[:2500], C)
    fsc, vsc = stored(X[2500:], "fp8")
    from oracle import formats
    _, e = formats.pack_e4m3(X[2500:])
    assert (e == 0).any() and (e == 1).any() and (e >= 2).any()
    res = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_LP))
    _, ref = oracle_mn(vfit, y[:2500], C, vsc)
    compare(res, ref)
    # without any recheck of near-ties, the e >= 2 rows are still recomputed in FP64
    off = to_np(nb.score(model, fsc, recheck=nb.NB_RECHECK_OFF))
    assert off["n_rechecked"] >= int((e >= 2).sum())
    rows = np.nonzero(e >= 2)[0]
    compare({k: (v[rows] if isinstance(v, np.ndarray) else v) for k, v in off.items()},
            {k: (v[rows] if isinstance(v, np.ndarray) else v) for k, v in ref.items()})


def test_tensor_scorer_bf16_values_outside_the_count_check():
    # fractional, tiny, negative-free large and out-of-range BF16 values: the
    # converters send their rows to the FP64 recheck, so the results still
    # equal the oracle on the stored values, in every recheck mode
    C, F = 6, 256
    X, y, _ = count_matrix(1170, 3400, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X[:3000], y[:3000], C)
    Xs = X[3000:].astype(np.float64)
    odd = {0: 0.5, 1: 1e-30, 2: 1500.0, 3: 1023.0, 5: 3e-6, 6: 70000.0, 7: 2.75}
    for r, v in odd.items():
        Xs[r, (7 * r) % F] = v
    fsc, vsc = stored(Xs, "bf16")
    _, ref = oracle_mn(vfit, y[:3000], C, vsc)
    for mode in (nb.NB_RECHECK_OFF, nb.NB_RECHECK_LABEL, nb.NB_RECHECK_LP):
        res = to_np(nb.score(model, fsc, recheck=mode))
        flagged = [r for r in odd if r != 3]
        assert res["n_rechecked"] >= len(flagged), (mode, res["n_rechecked"])
        compare(res, ref, check_lp=mode == nb.NB_RECHECK_LP)


@pytest.mark.parametrize("fmt", ["u8", "u8ovf", "bf16", "fp8"])
def test_tensor_scorer_empty_and_single_row(fmt):
    # no rows, one row (a single ragged tile), and 129 rows (one full tile and
    # one row of the next)
    C, F = 5, 300
    X, y, _ = count_matrix(1190, 3000, F, C=C, conc=0.1, clip=255)
    model, vfit = _model("u8", X, y, C)
    e, _ = stored(X[:0], fmt)
    r0 = nb.score(model, e)
    assert r0["label"].numel() == 0 and int(r0["n_rechecked"].item()) == 0
    for n in (1, 129):
        f, v = stored(X[:n], fmt)
        assert nb.score_path(model, f) == nb.NB_PATH_TENSOR
        res = to_np(nb.score(model, f, recheck=nb.NB_RECHECK_LP))
        _, ref = oracle_mn(vfit, y, C, v)
        compare(res, ref)
