"""Pins of the group-wise oracle (size groups, small-group fallback, top-k
opcode selection, the whole per-group method) against what the paper prints
and what the definitions fix, independently of the oracle's own code."""
import itertools

import numpy as np
import pytest

from oracle import groupwise as gw
from oracle import mn_fit, score


# ---------------------------------------------------------------- size groups
def test_size_group_boundaries():
    # Sec. 3: 100 groups of 5 KB each below 500 KB
    sizes = [0, 1, 5119, 5120, 10239, 10240, 500 * 1024 - 1, 500 * 1024, 10**9]
    assert gw.size_group(sizes).tolist() == [0, 0, 0, 1, 1, 2, 99, 99, 99]
    assert gw.size_group([99, 100, 250], bin_bytes=100, n_bins=3).tolist() == [0, 1, 2]
    with pytest.raises(ValueError):
        gw.size_group([-1])


# -------------------------------------------------------- small-group fallback
def test_group_models_paper_example():
    # Sec. 4 names the 5th, 8th, 61st, 65th, 97th, 98th and 100th groups (one
    # based) as having fewer than six files of a class.
    untrained = {5, 8, 61, 65, 97, 98, 100}
    cc = np.full((100, 2), 40)
    for g in untrained:
        cc[g - 1] = (3, 50)
    m = gw.group_models(cc)
    one_based = {g: int(m[g - 1]) + 1 for g in range(1, 101)}
    assert one_based[5] == 6 and one_based[8] == 9
    assert one_based[61] == 62 and one_based[65] == 66
    assert one_based[97] == 99 and one_based[98] == 99     # next trained above
    assert one_based[100] == 99                             # none above: below
    for g in set(range(1, 101)) - untrained:
        assert one_based[g] == g


def test_group_models_threshold_and_edges():
    cc = np.array([[6, 5], [6, 6], [0, 0], [100, 5]])
    assert gw.group_models(cc).tolist() == [1, 1, 1, 1]
    assert gw.group_models(cc, min_files=5).tolist() == [0, 1, 3, 3]
    only_first = np.zeros((5, 2), np.int64)
    only_first[0] = (7, 7)
    assert gw.group_models(only_first).tolist() == [0, 0, 0, 0, 0]
    with pytest.raises(ValueError):
        gw.group_models(np.zeros((4, 2)))


# ---------------------------------------------------------- feature selection
def test_select_hand_worked_total_norm():
    # f0 = [2,0,3,1]/6, f1 = [1,4,1,2]/8 -> |f1 - f0| = [5, 12, 9, 2] / 24
    N = np.array([[2, 0, 3, 1], [1, 4, 1, 2]])
    assert gw.select_features(N, (2, 4), 4).tolist() == [1, 2, 0, 3]
    assert gw.select_features(N, (2, 4), 2).tolist() == [1, 2]


def test_select_hand_worked_files_norm():
    # f0 = [2,0,3,1]/2, f1 = [1,4,1,2]/4 -> |f1 - f0| = [3, 4, 5, 0] / 4
    N = np.array([[2, 0, 3, 1], [1, 4, 1, 2]])
    assert gw.select_features(N, (2, 4), 4, norm="files").tolist() == [2, 1, 0, 3]


def test_select_ties_go_to_lower_index():
    # f0 = [1/2, 1/2, 0], f1 = [0, 0, 1] -> [1/2, 1/2, 1]
    N = np.array([[1, 1, 0], [0, 0, 2]])
    assert gw.select_features(N, (1, 1), 3).tolist() == [2, 0, 1]
    # identical profiles: every score 0, the index order remains
    P = np.array([[3, 1, 4, 1], [6, 2, 8, 2]])
    assert gw.select_features(P, (1, 2), 4).tolist() == [0, 1, 2, 3]


def test_select_empty_class():
    # a class with no counts has f = 0: the ranking follows the other class
    N = np.array([[5, 9, 1, 9], [0, 0, 0, 0]])
    assert gw.select_features(N, (3, 0), 4).tolist() == [1, 3, 0, 2]
    assert gw.select_features(N, (3, 0), 4, norm="files").tolist() == [1, 3, 0, 2]


def test_select_matches_float_ranking_when_keys_are_well_separated():
    # an independent library ranking: numpy lexsort on FP64 keys, used only
    # where the FP64 keys are far apart relative to their rounding error
    rng = np.random.default_rng(11)
    for _ in range(20):
        F = int(rng.integers(5, 300))
        N = rng.integers(0, 5000, size=(2, F)).astype(np.uint64)
        nf = rng.integers(1, 50, size=2)
        for norm in gw.NORMS:
            D = N.sum(axis=1).astype(np.float64) if norm == "total" else nf.astype(np.float64)
            key = np.abs(N[1] / D[1] - N[0] / D[0])
            s = np.sort(key)
            gaps = np.diff(s)
            if gaps.size and gaps.min() <= 1e-12 * max(1.0, s.max()):
                continue
            k = int(rng.integers(1, F + 1))
            ref = np.lexsort((np.arange(F), -key))[:k]
            assert gw.select_features(N, nf, k, norm).tolist() == ref.tolist()


def test_select_brute_force_top_sets():
    # every k-subset of a tiny group: the selected set has the largest score
    # sum, and among equal sums the lexicographically smallest sorted indices
    rng = np.random.default_rng(12)
    for _ in range(40):
        F = int(rng.integers(1, 6))
        N = rng.integers(0, 4, size=(2, F))
        nf = rng.integers(1, 4, size=2)
        sc = gw.feature_scores(N, nf, "total")
        for k in range(1, F + 1):
            best = max(itertools.combinations(range(F), k),
                       key=lambda S: (sum(sc[j] for j in S), [-j for j in S]))
            got = gw.select_features(N, nf, k)
            assert sorted(got.tolist()) == list(best)


def test_select_invariances():
    rng = np.random.default_rng(13)
    F = 64
    N = rng.integers(0, 10**6, size=(2, F)).astype(np.uint64)
    nf = np.array([10, 17])
    sel = gw.select_features(N, nf, 20)
    # classes swapped: |f1 - f0| is symmetric
    assert gw.select_features(N[::-1], nf[::-1], 20).tolist() == sel.tolist()
    # a class's counts scaled by an integer: its distribution is unchanged
    N2 = N.copy()
    N2[0] *= np.uint64(7)
    assert gw.select_features(N2, nf, 20).tolist() == sel.tolist()
    # features permuted: the same opcodes are chosen (keys here are distinct)
    perm = rng.permutation(F)
    selp = gw.select_features(N[:, perm], nf, 20)
    assert perm[selp].tolist() == sel.tolist()


def test_select_rejects_bad_k():
    N = np.ones((2, 4), np.int64)
    for k in (0, 5):
        with pytest.raises(ValueError):
            gw.select_features(N, (1, 1), k)


# ------------------------------------------------------------- whole method
def _groups_data(seed, n, F, bins):
    rng = np.random.default_rng(seed)
    y = rng.integers(0, 2, n).astype(np.int32)
    p = rng.dirichlet(np.full(F, 0.3), size=2)
    X = np.stack([rng.multinomial(int(t), p[c]) for t, c in
                  zip(rng.integers(50, 400, n), y)]).astype(np.uint16)
    sizes = rng.integers(0, bins * 5120, n)
    return X, y, sizes


def test_one_group_all_features_is_plain_naive_bayes():
    # k = F and every file in one group: the method reduces to one model on all
    # features (columns reordered, so scores agree to rounding)
    X, y, _ = _groups_data(21, 400, 12, 1)
    sizes = np.full(400, 777)
    fitted = gw.fit_groups(X, y, sizes, k=12)
    assert set(fitted["models"]) == {0}
    res = gw.score_groups(X, sizes, fitted)
    ref = score(X.astype(np.float64), mn_fit(X, y, 2))
    assert (res["label"] == ref["label"]).all()
    assert np.allclose(res["lp"], ref["lp"], rtol=0, atol=1e-9)


def test_fallback_files_use_the_next_trained_groups_model():
    X, y, sizes = _groups_data(22, 900, 16, 6)
    # empty the 3rd group of benign files: it is untrained and falls back to 4
    g = gw.size_group(sizes)
    keep = ~((g == 2) & (y == 0))
    fitted = gw.fit_groups(X[keep], y[keep], sizes[keep], k=8)
    assert fitted["model_of"][2] == 3 and 2 not in fitted["models"]
    test = np.nonzero(g == 2)[0]
    res = gw.score_groups(X[test], sizes[test], fitted)
    assert (res["model"] == 3).all()
    cols = fitted["cols"][3]
    ref = score(X[test][:, cols].astype(np.float64), fitted["models"][3])
    assert (res["label"] == ref["label"]).all()
    # bins past the trained range fall back downward
    assert fitted["model_of"][99] == 5
