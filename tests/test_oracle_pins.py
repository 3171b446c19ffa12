"""Pins for the FP64 oracle against things other than itself.

Each test checks the oracle (oracle/) against what the paper and the
mathematics fix: hand-worked examples in exact rationals, brute force over
exact normalised products of likelihoods, high-precision density products,
an independent library implementation, invariants and closed forms.  Each is
chosen so that a plausible slip in the oracle (a dropped smoothing term, a
wrong sign, a transposed table, an off-by-one feature, a tie sent the wrong
way) fails at least one of them.  Posterior and decision rule: Sec. 4.
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------
# Hand-worked examples (exact rationals)
# ----------------------------------------------------------------------------
def test_handworked_multinomial(golden_dir):
    g = _load(golden_dir, "handworked_multinomial.json")
    X = np.array(g["train_X"], float)
    y = np.array(g["train_y"])
    m = oracle.mn_fit(X, y, 2, alpha=g["alpha"], log_prior=np.log([0.5, 0.5]))
    assert m["counts"].tolist() == g["counts"]
    assert m["nc"].tolist() == g["nc"]
    for c in range(2):
        for j in range(3):
            th = Fraction(g["theta"][c][j])
            assert m["log_theta"][c, j] == pytest.approx(math.log(th), rel=0, abs=1e-15)
    xs = np.array([case["x"] for case in g["cases"]], float)
    r = oracle.score(xs, m)
    for i, case in enumerate(g["cases"]):
        j0, j1 = (Fraction(v) for v in case["joint"])
        assert r["s"][i, 0] == pytest.approx(math.log(j0), abs=1e-14)
        assert r["s"][i, 1] == pytest.approx(math.log(j1), abs=1e-14)
        pm = Fraction(case["posterior_malware"])
        assert math.exp(r["lp"][i, 1]) == pytest.approx(float(pm), abs=1e-15)
        assert math.exp(r["lp"][i, 0]) == pytest.approx(float(1 - pm), abs=1e-15)
        assert int(r["label"][i]) == case["label"]
        assert r["margin"][i] == pytest.approx(abs(math.log(j1 / j0)), abs=1e-14)


def test_handworked_multinomial_empirical_prior(golden_dir):
    # two files per class -> empirical prior 1/2: same result as the given prior
    g = _load(golden_dir, "handworked_multinomial.json")
    X = np.array(g["train_X"], float)
    y = np.array(g["train_y"])
    m = oracle.mn_fit(X, y, 2, alpha=1)
    assert np.allclose(m["log_pi"], np.log(0.5), atol=0, rtol=1e-15)


def test_handworked_gaussian(golden_dir):
    g = _load(golden_dir, "handworked_gaussian.json")
    X = np.array(g["train_X"], float)
    y = np.array(g["train_y"])
    m = oracle.gauss_fit(X, y, 2, var_smoothing=0.0, log_prior=np.log([0.5, 0.5]))
    assert m["mu"].tolist() == g["mu"]
    assert m["var"].tolist() == g["var"]
    case = g["cases"][0]
    r = oracle.score(np.array([case["x"]], float), m)
    l2p = math.log(2 * math.pi)
    s0 = math.log(0.5) - 0.5 * (3 * l2p + case["quad"][0])
    s1 = math.log(0.5) - 0.5 * (3 * l2p + math.log(4) + case["quad"][1])
    assert r["s"][0, 0] == pytest.approx(s0, abs=1e-14)
    assert r["s"][0, 1] == pytest.approx(s1, abs=1e-14)
    assert r["margin"][0] == pytest.approx(0.5 * (9 - 5.25 - math.log(4)), abs=1e-14)
    assert int(r["label"][0]) == case["label"]


# ----------------------------------------------------------------------------
# Brute force: exact normalised products of likelihoods
# ----------------------------------------------------------------------------
def _exact_posterior(Xtr, ytr, C, alpha, x, prior=None):
    n, F = Xtr.shape
    joints = []
    for c in range(C):
        rows = Xtr[ytr == c]
        Ncj = [int(rows[:, j].sum()) for j in range(F)]
        Nc = sum(Ncj)
        pc = Fraction(len(rows), n) if prior is None else prior[c]
        p = pc
        for j in range(F):
            p *= Fraction(Ncj[j] + alpha, Nc + alpha * F) ** int(x[j])
        joints.append(p)
    tot = sum(joints)
    return joints, [jc / tot for jc in joints]


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_rational_multinomial(seed):
    rng = np.random.default_rng(1000 + seed)
    C = int(rng.integers(2, 4))
    F = int(rng.integers(1, 5))
    alpha = int(rng.integers(1, 3))
    n = int(rng.integers(C, 3 * C + 3))
    y = np.concatenate([np.arange(C), rng.integers(0, C, size=n - C)]).astype(np.int32)
    Xtr = rng.integers(0, 6, size=(n, F)).astype(float)
    Xte = rng.integers(0, 6, size=(6, F)).astype(float)
    m = oracle.mn_fit(Xtr, y, C, alpha=alpha)
    r = oracle.score(Xte, m)
    for i in range(Xte.shape[0]):
        joints, post = _exact_posterior(Xtr, y, C, alpha, Xte[i])
        for c in range(C):
            assert abs(math.exp(r["lp"][i, c]) - float(post[c])) <= 1e-14
        best = max(range(C), key=lambda c: (joints[c], -c))
        assert int(r["label"][i]) == best
        order = sorted(joints, reverse=True)
        if order[1] > 0:
            exact_margin = math.log(order[0].numerator * order[1].denominator) - \
                math.log(order[0].denominator * order[1].numerator)
            assert r["margin"][i] == pytest.approx(exact_margin, abs=1e-12)


def test_bruteforce_counts_enumerated():
    # every 2-file, 2-feature training set with counts 0..2: counts and n_c exact
    vals = range(3)
    for a, b, c, d in itertools.product(vals, repeat=4):
        X = np.array([[a, b], [c, d], [1, 0]], float)
        y = np.array([0, 1, 1])
        m = oracle.mn_fit(X, y, 2)
        assert m["counts"].tolist() == [[a, b], [c + 1, d]]
        assert m["nc"].tolist() == [1, 2]


# ----------------------------------------------------------------------------
# Gaussian: exact moments and a high-precision product of densities
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(10))
def test_gaussian_exact_moments_and_density_product(seed):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    rng = np.random.default_rng(2000 + seed)
    C, F = 3, int(rng.integers(1, 5))
    n = 12
    y = np.array([i % C for i in range(n)], np.int32)
    while True:   # redraw until no class has a constant feature
        X = rng.integers(-20, 21, size=(n, F)).astype(float)
        if all((X[y == c].var(axis=0) > 0).all() for c in range(C)):
            break
    m = oracle.gauss_fit(X, y, C, var_smoothing=0.0)
    for c in range(C):
        rows = X[y == c]
        for j in range(F):
            mu = Fraction(int(rows[:, j].sum()), len(rows))
            var = sum((Fraction(int(v)) - mu) ** 2 for v in rows[:, j]) / len(rows)
            assert m["mu"][c, j] == pytest.approx(float(mu), rel=1e-15, abs=1e-15)
            assert m["var"][c, j] == pytest.approx(float(var), rel=1e-14)
    Xte = rng.normal(0, 8, size=(5, F))
    r = oracle.score(Xte, m)
    for i in range(Xte.shape[0]):
        dens = []
        for c in range(C):
            rows = X[y == c]
            p = mpmath.mpf(len(rows)) / n
            for j in range(F):
                mu = mpmath.mpf(int(rows[:, j].sum())) / len(rows)
                var = sum((mpmath.mpf(int(v)) - mu) ** 2 for v in rows[:, j]) / len(rows)
                xx = mpmath.mpf(float(Xte[i, j]))
                p *= mpmath.exp(-(xx - mu) ** 2 / (2 * var)) / mpmath.sqrt(2 * mpmath.pi * var)
            dens.append(p)
        tot = sum(dens)
        for c in range(C):
            assert abs(math.exp(r["lp"][i, c]) - float(dens[c] / tot)) <= 1e-13
            assert r["s"][i, c] == pytest.approx(float(mpmath.log(dens[c])), rel=1e-13, abs=1e-12)


def test_gaussian_var_smoothing_epsilon():
    rng = np.random.default_rng(7)
    X = rng.normal(size=(50, 4)) * np.array([1.0, 3.0, 0.5, 2.0])
    y = (np.arange(50) % 2).astype(np.int32)
    m0 = oracle.gauss_fit(X, y, 2, var_smoothing=0.0)
    m1 = oracle.gauss_fit(X, y, 2, var_smoothing=1e-3)
    eps = 1e-3 * X.var(axis=0).max()
    assert np.allclose(m1["var"] - m0["var"], eps, rtol=1e-9, atol=0)


# ----------------------------------------------------------------------------
# Independent library implementation (special case reducing to a library)
# ----------------------------------------------------------------------------
def test_against_sklearn_multinomial():
    nb = pytest.importorskip("sklearn.naive_bayes")
    rng = np.random.default_rng(11)
    C, F, n = 4, 37, 300
    y = np.concatenate([np.arange(C), rng.integers(0, C, n - C)]).astype(np.int32)
    prof = rng.dirichlet(np.full(F, 0.3), size=C)
    X = np.stack([rng.multinomial(int(rng.integers(1, 400)), prof[c]) for c in y]).astype(float)
    clf = nb.MultinomialNB(alpha=1.0).fit(X, y)
    m = oracle.mn_fit(X, y, C, alpha=1.0)
    assert np.allclose(m["log_theta"], clf.feature_log_prob_, rtol=1e-13, atol=1e-13)
    assert np.allclose(m["log_pi"], clf.class_log_prior_, rtol=1e-13, atol=1e-13)
    Xte = np.stack([rng.multinomial(int(rng.integers(0, 400)), prof[c])
                    for c in rng.integers(0, C, 200)]).astype(float)
    r = oracle.score(Xte, m)
    assert np.allclose(r["s"], clf.predict_joint_log_proba(Xte), rtol=1e-12, atol=1e-9)
    assert np.allclose(r["lp"], clf.predict_log_proba(Xte), rtol=1e-9, atol=1e-9)
    assert (r["label"] == clf.predict(Xte)).all()


def test_against_sklearn_gaussian():
    nb = pytest.importorskip("sklearn.naive_bayes")
    import synth
    w = synth.gaussian_workload(5, F=16, n_fit_per_class=200, n_score_per_class=300)
    clf = nb.GaussianNB(var_smoothing=1e-9, priors=[0.5, 0.5]).fit(
        w["X_fit"].astype(float), w["y_fit"])
    m = oracle.gauss_fit(w["X_fit"], w["y_fit"], 2, var_smoothing=1e-9,
                         log_prior=np.log([0.5, 0.5]))
    assert np.allclose(m["mu"], clf.theta_, rtol=1e-12, atol=1e-12)
    assert np.allclose(m["var"], clf.var_, rtol=1e-12, atol=0)
    Xte = w["X_score"].astype(float)
    r = oracle.score(Xte, m)
    assert np.allclose(r["s"], clf.predict_joint_log_proba(Xte), rtol=1e-11, atol=1e-9)
    assert (r["label"] == clf.predict(Xte)).all()


# ----------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------
def _random_mn(seed, C=3, F=20, n=120):
    rng = np.random.default_rng(seed)
    y = np.concatenate([np.arange(C), rng.integers(0, C, n - C)]).astype(np.int32)
    prof = rng.dirichlet(np.full(F, 0.2), size=C)
    X = np.stack([rng.multinomial(int(rng.integers(0, 500)), prof[c]) for c in y]).astype(float)
    Xte = np.stack([rng.multinomial(int(rng.integers(0, 500)), prof[c])
                    for c in rng.integers(0, C, 60)]).astype(float)
    return X, y, Xte


def test_posteriors_sum_to_one():
    X, y, Xte = _random_mn(1)
    r = oracle.score(Xte, oracle.mn_fit(X, y, 3))
    assert np.allclose(np.exp(r["lp"]).sum(axis=1), 1.0, atol=1e-12, rtol=0)
    assert (r["margin"] >= 0).all()


def test_count_totals_exact():
    X, y, _ = _random_mn(2)
    m = oracle.mn_fit(X, y, 3)
    assert int(m["counts"].sum()) == int(X.sum())
    assert int(m["nc"].sum()) == X.shape[0]
    for c in range(3):
        assert m["counts"][c].tolist() == X[y == c].sum(axis=0).astype(int).tolist()


def test_feature_permutation_invariance():
    X, y, Xte = _random_mn(3)
    perm = np.random.default_rng(0).permutation(X.shape[1])
    r0 = oracle.score(Xte, oracle.mn_fit(X, y, 3))
    m1 = oracle.mn_fit(X[:, perm], y, 3)
    r1 = oracle.score(Xte[:, perm], m1)
    assert (r0["label"] == r1["label"]).all()
    assert np.allclose(r0["s"], r1["s"], rtol=1e-12, atol=1e-9)


def test_file_permutation_invariance():
    X, y, Xte = _random_mn(4)
    perm = np.random.default_rng(1).permutation(X.shape[0])
    m0 = oracle.mn_fit(X, y, 3)
    m1 = oracle.mn_fit(X[perm], y[perm], 3)
    assert (m0["counts"] == m1["counts"]).all()
    assert (m0["log_theta"] == m1["log_theta"]).all()
    assert (m0["log_pi"] == m1["log_pi"]).all()


def test_duplicate_training_set_doubles_alpha():
    X, y, Xte = _random_mn(5)
    m0 = oracle.mn_fit(X, y, 3, alpha=1.0)
    m1 = oracle.mn_fit(np.concatenate([X, X]), np.concatenate([y, y]), 3, alpha=2.0)
    assert np.allclose(m0["log_theta"], m1["log_theta"], rtol=0, atol=1e-14)
    assert np.allclose(m0["log_pi"], m1["log_pi"], rtol=0, atol=1e-15)


# ----------------------------------------------------------------------------
# Special cases with closed forms
# ----------------------------------------------------------------------------
def test_single_feature_closed_form():
    # F = 1: theta = (N + a)/(N + a) = 1 for every class, so only the prior decides
    X = np.array([[3.0], [5.0], [1.0], [0.0], [2.0]])
    y = np.array([0, 1, 1, 1, 0])
    m = oracle.mn_fit(X, y, 2, alpha=1.0)
    assert np.allclose(m["log_theta"], 0.0, atol=1e-15)
    r = oracle.score(np.array([[0.0], [7.0], [100.0]]), m)
    assert (r["label"] == 1).all()                       # prior 3/5 > 2/5
    assert np.allclose(r["margin"], math.log(1.5), atol=1e-15)


def test_identical_profiles_prior_decides():
    X = np.array([[1, 2, 3], [1, 2, 3], [1, 2, 3], [1, 2, 3]], float)
    y = np.array([0, 1, 1, 1])
    # per-class counts differ by scale only; without smoothing (alpha = 0)
    # theta is identical, so the prior alone decides
    m = oracle.mn_fit(X, y, 2, alpha=0.0)
    assert np.allclose(m["log_theta"][0], m["log_theta"][1], atol=1e-15)
    r = oracle.score(np.array([[9, 0, 0], [0, 0, 9]], float), m)
    assert (r["label"] == 1).all()
    m2 = oracle.mn_fit(X, y, 2, alpha=0.0, log_prior=np.log([0.5, 0.5]))
    r2 = oracle.score(np.array([[9, 0, 0]], float), m2)
    assert r2["margin"][0] <= 1e-12          # a tie up to rounding of log theta


def test_all_zero_row_tie_goes_to_benign():
    X, y, _ = _random_mn(6, C=2)
    m = oracle.mn_fit(X, y, 2, log_prior=np.log([0.5, 0.5]))
    r = oracle.score(np.zeros((1, X.shape[1])), m)
    assert int(r["label"][0]) == 0 and r["margin"][0] == 0.0
    assert np.allclose(r["lp"][0], math.log(0.5), atol=1e-15)


def test_two_class_softplus_form():
    X, y, Xte = _random_mn(7, C=2)
    m = oracle.mn_fit(X, y, 2)
    r = oracle.score(Xte, m)
    d = r["s"][:, 1] - r["s"][:, 0]
    assert np.allclose(r["lp"][:, 1], -np.logaddexp(0, -d), rtol=1e-12, atol=1e-12)
    assert np.allclose(r["lp"][:, 0], -np.logaddexp(0, d), rtol=1e-12, atol=1e-12)
    assert np.allclose(r["margin"], np.abs(d), rtol=1e-12, atol=1e-9)
    assert (r["label"] == (d > 0)).all()


def test_gaussian_equal_variance_is_linear_discriminant():
    rng = np.random.default_rng(12)
    F = 5
    mu0, mu1 = rng.normal(size=F), rng.normal(size=F)
    var = rng.uniform(0.5, 2.0, size=F)
    m = {"kind": "gaussian", "mu": np.stack([mu0, mu1]), "var": np.stack([var, var]),
         "log_pi": np.log([0.3, 0.7])}
    Xte = rng.normal(size=(40, F))
    r = oracle.score(Xte, m)
    w = (mu1 - mu0) / var
    b = math.log(0.7 / 0.3) - 0.5 * np.sum((mu1 ** 2 - mu0 ** 2) / var)
    d = Xte @ w + b
    assert np.allclose(r["s"][:, 1] - r["s"][:, 0], d, rtol=1e-12, atol=1e-12)


def test_rejects_bad_inputs():
    with pytest.raises(oracle.OracleError):
        oracle.mn_fit(np.array([[1.5, 0.0]]), np.array([0]), 2, log_prior=[0.0, 0.0])
    with pytest.raises(oracle.OracleError):
        oracle.mn_fit(np.array([[1.0, 0.0]]), np.array([0]), 2)   # class 1 empty
    with pytest.raises(oracle.OracleError):
        oracle.mn_fit(np.array([[-1.0, 0.0]]), np.array([0]), 2, log_prior=[0.0, 0.0])
