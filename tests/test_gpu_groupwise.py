"""The group-wise method on the GPU (Sec. 3 size groups and top-k opcodes,
Sec. 4 per-group models and the small-group rule) against the oracle: routing
and its stable order, the exact top-k ranking, the column gather (all
bit-exact), and whole-pipeline labels / log posteriors over up to 100
models scored in one launch."""
import numpy as np
import pytest
import torch

import synth
from oracle import groupwise as ogw
from oracle import mn_fit, score as oscore
from tests._common import compare, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    nb.build()
    nb.lib()


def _sizes(seed, n, hi=600 * 1024):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, hi, n).astype(np.int64)
    if n > 3:
        s[:3] = [0, 512000, 10**9]           # first group, the 500 KB edge, far beyond
    return s


# -------------------------------------------------------------------- routing
@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 10007, 70001])
def test_route_groups_and_stable_order(n):
    s = _sizes(100 + n, n)
    y = np.random.default_rng(n).integers(0, 2, n).astype(np.int32)
    r = nb.route(torch.from_numpy(s).cuda(), y=torch.from_numpy(y).cuda() if n else None)
    torch.cuda.synchronize()
    g_ref = ogw.size_group(s)
    assert r["status"].item() == 0
    assert (r["group"].cpu().numpy() == g_ref).all()
    # counting sort, stable: numpy's stable argsort of the groups
    assert (r["order"].cpu().numpy() == np.argsort(g_ref, kind="stable")).all()
    offs = r["offsets"].cpu().numpy()
    assert (offs == np.concatenate([[0], np.cumsum(np.bincount(g_ref, minlength=100))])).all()
    if n:
        cc = r["class_counts"].cpu().numpy()
        assert (cc == ogw.group_class_counts(g_ref, y)).all()


@pytest.mark.parametrize("n_bins,bin_bytes", [(1, 5120), (512, 1000), (333, 7)])
def test_route_group_count_extremes(n_bins, bin_bytes):
    # one group, the most groups a route takes (512: two scan slices per
    # group), and a count that does not divide the 1,024 scan threads
    n = 20000
    s = np.random.default_rng(n_bins).integers(0, bin_bytes * (n_bins + 3), n).astype(np.int64)
    r = nb.route(torch.from_numpy(s).cuda(), bin_bytes=bin_bytes, n_bins=n_bins)
    g = ogw.size_group(s, bin_bytes, n_bins)
    assert (r["group"].cpu().numpy() == g).all()
    assert (r["order"].cpu().numpy() == np.argsort(g, kind="stable")).all()
    offs = r["offsets"].cpu().numpy()
    assert (offs == np.concatenate([[0], np.cumsum(np.bincount(g, minlength=n_bins))])).all()


def test_route_through_a_model_map():
    n = 30000
    s = _sizes(7, n)
    cc = np.full((100, 2), 50)
    cc[[4, 7, 60, 64, 96, 97, 99]] = (2, 40)
    mo_bins = nb.group_fallback(cc)
    assert mo_bins.tolist() == ogw.group_models(cc).tolist()
    trained = sorted(set(mo_bins.tolist()))
    slot = np.array([trained.index(m) for m in mo_bins], np.int32)
    r = nb.route(torch.from_numpy(s).cuda(), model_of=slot, n_groups=len(trained))
    ref_g = slot[ogw.size_group(s)]
    assert (r["group"].cpu().numpy() == ref_g).all()
    assert (r["order"].cpu().numpy() == np.argsort(ref_g, kind="stable")).all()


def test_group_fallback_host_rules():
    with pytest.raises(nb.NbError):
        nb.group_fallback(np.zeros((5, 2)))
    cc = np.array([[6, 5], [6, 6], [0, 0], [100, 5]])
    assert nb.group_fallback(cc).tolist() == ogw.group_models(cc).tolist()
    assert nb.group_fallback(cc, 5).tolist() == ogw.group_models(cc, 5).tolist()


def test_route_flags_negative_sizes():
    s = np.array([5, -1, 7000], np.int64)
    r = nb.route(torch.from_numpy(s).cuda())
    assert r["status"].item() & nb.ST_BAD_ROUTE
    assert r["group"].cpu().tolist() == [0, 0, 1]          # counted as size 0


# ---------------------------------------------------------- feature selection
def _two_class_group(seed, n, F, ties=False, empty_class=False):
    rng = np.random.default_rng(seed)
    X = rng.poisson(rng.gamma(0.3, 8.0, size=F), size=(n, F)).clip(0, 255).astype(np.uint8)
    y = (np.arange(n) % 2).astype(np.int32)
    if ties:
        X[:, 5] = X[:, 3]                       # identical columns: equal keys
        X[:, F - 1] = X[:, 0]
    if empty_class:
        X[y == 1] = 0                           # class 1 has no counts at all
    return X, y


@pytest.mark.parametrize("F,k", [(64, 1), (64, 64), (1000, 20), (1500, 200), (3000, 160)])
@pytest.mark.parametrize("norm", [nb.NB_SELECT_TOTAL, nb.NB_SELECT_FILES])
def test_select_matches_oracle_exactly(F, k, norm):
    models, refs = [], []
    for i in range(3):
        X, y = _two_class_group(1000 + F + i, 300 + 17 * i, F, ties=(i == 1),
                                empty_class=(i == 2))
        Xd = torch.zeros((X.shape[0], (F + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
        Xd[:, :F] = torch.from_numpy(X).cuda()
        models.append(nb.fit(Xd[:, :F], torch.from_numpy(y).cuda(), 2))
        m = mn_fit(X, y, 2)                      # oracle counts, not the GPU's
        refs.append(ogw.select_features(m["counts"], m["nc"], k,
                                        "total" if norm == nb.NB_SELECT_TOTAL else "files"))
    cols = nb.select_features(models, k, norm).cpu().numpy()
    for i in range(3):
        assert cols[i].tolist() == refs[i].tolist(), f"model {i}"


# ------------------------------------------------------------------- gather
@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_gather_rows_and_columns(dt):
    rng = np.random.default_rng(31)
    n, F, G, k = 5003, 700, 9, 77
    X = rng.integers(0, 256, size=(n, F))
    X = X.astype(np.uint8) if dt == "u8" else (X * 1.5).astype(np.float32)
    order = rng.permutation(n).astype(np.int64)
    group = rng.integers(0, G, n).astype(np.int32)
    cols = np.stack([rng.choice(F, k, replace=False) for _ in range(G)]).astype(np.int32)
    Xd = torch.from_numpy(X).cuda()
    out, st = nb.gather(Xd, torch.from_numpy(cols).cuda(), order=torch.from_numpy(order).cuda(),
                        group=torch.from_numpy(group).cuda(), n_groups=G)
    got = out.cpu().numpy()
    ref = np.stack([X[order[r], cols[group[order[r]]]] for r in range(n)])
    assert st.item() == 0
    assert (got == ref).all()
    full = out.as_strided((n, nb.padded_ld(k, nb.NB_U8 if dt == "u8" else nb.NB_F32)),
                          (out.stride(0), 1)).cpu().numpy()
    assert (full[:, k:] == 0).all()             # padding is zero


def test_gather_bad_group_and_column_give_zeros_and_status():
    X = torch.arange(40, dtype=torch.uint8, device="cuda").reshape(4, 10)
    cols = torch.tensor([[1, 2, 99]], dtype=torch.int32, device="cuda")
    group = torch.tensor([0, 3, 0, 0], dtype=torch.int32, device="cuda")
    out, st = nb.gather(X, cols, group=group, n_groups=1)
    got = out.cpu().numpy()
    assert st.item() & nb.ST_BAD_ROUTE
    assert got[1].tolist() == [0, 0, 0]
    assert got[0].tolist() == [1, 2, 0]
    # a source row outside the matrix
    order = torch.tensor([3, 7], dtype=torch.int64, device="cuda")
    out, st = nb.gather(X, cols[:, :2], order=order)
    assert st.item() & nb.ST_BAD_ROUTE
    assert out.cpu().numpy().tolist() == [[31, 32], [0, 0]]


# -------------------------------------------------------------- whole method
def _workload(seed, n, F, n_bins):
    X, y, s = synth.groupwise_workload(seed, n, F, n_bins=n_bins)
    return X.numpy(), y, s


def _fit_both(X, y, s, k, norm, n_bins):
    fitted_o = ogw.fit_groups(X, y, s, k, "total" if norm == nb.NB_SELECT_TOTAL else "files",
                              n_bins=n_bins)
    Xd = torch.zeros((X.shape[0], (X.shape[1] + 15) // 16 * 16), dtype=torch.uint8,
                     device="cuda")
    Xd[:, :X.shape[1]] = torch.from_numpy(X).cuda()
    fitted_g = nb.fit_groupwise(Xd[:, :X.shape[1]], torch.from_numpy(y).cuda(),
                                torch.from_numpy(s).cuda(), k, norm, n_bins=n_bins)
    return fitted_o, fitted_g


@pytest.mark.parametrize("k,norm", [(20, nb.NB_SELECT_TOTAL), (64, nb.NB_SELECT_FILES)])
def test_groupwise_pipeline_matches_oracle(k, norm):
    n_bins, F = 24, 256
    X, y, s = _workload(41, 9000, F, n_bins)
    tr, te = synth.split_per_class(42, y)
    fo, fg = _fit_both(X[tr], y[tr], s[tr], k, norm, n_bins)
    # same trained groups, same fallback, same opcodes
    assert fg["groups"] == sorted(fo["models"])
    assert [fg["groups"][m] for m in fg["model_of"]] == fo["model_of"].tolist()
    for i, g in enumerate(fg["groups"]):
        assert fg["cols"][i].cpu().tolist() == fo["cols"][g].tolist(), f"group {g}"
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=len(te),
                      bin_bytes=nb.BIN_BYTES)
    Xt = torch.zeros((len(te), 256), dtype=torch.uint8, device="cuda")
    Xt[:] = torch.from_numpy(X[te]).cuda()
    res = gw.classify(Xt, torch.from_numpy(s[te]).cuda())
    torch.cuda.synchronize()
    assert gw.status() == 0
    ref = ogw.score_groups(X[te], s[te], fo)
    compare(to_np(res), ref)


def test_groupwise_one_hundred_models_in_one_launch():
    # every one of the 100 size groups trained: 100 models, one batched launch
    n_bins, F, k = 100, 128, 20
    rng = np.random.default_rng(51)
    per = 40
    s = (np.repeat(np.arange(n_bins), per) * 5120 + rng.integers(0, 5120, n_bins * per))
    y = np.tile(np.arange(per) % 2, n_bins).astype(np.int32)
    p = synth.dirichlet_profiles(52, 2 * n_bins, F, 0.2)
    T = np.full(n_bins * per, 600.0)
    X = synth.count_rows(53, p, (s // 5120) * 2 + y, T, 255, out_dtype="uint8").numpy()
    fo, fg = _fit_both(X, y, s.astype(np.int64), k, nb.NB_SELECT_TOTAL, n_bins)
    assert len(fg["models"]) == 100
    st = rng.integers(0, 100 * 5120, 20000).astype(np.int64)
    Xt_np = synth.count_rows(54, p, (st // 5120) * 2 + rng.integers(0, 2, 20000),
                             np.full(20000, 600.0), 255, out_dtype="uint8").numpy()
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=20000)
    launches0 = nb.nb_kernel_launches()
    res = gw.classify(torch.from_numpy(Xt_np).cuda(), torch.from_numpy(st).cuda())
    torch.cuda.synchronize()
    launches = nb.nb_kernel_launches() - launches0
    assert launches <= 2, launches                 # fused scorer + recheck
    compare(to_np(res), ogw.score_groups(Xt_np, st, fo))


def test_groupwise_rows_equal_single_group_scoring():
    # each file's result is its model's nb_score_group on its gathered row
    n_bins, F, k = 16, 192, 40
    X, y, s = _workload(61, 6000, F, n_bins)
    _, fg = _fit_both(X, y, s, k, nb.NB_SELECT_TOTAL, n_bins)
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=6000)
    Xd = torch.from_numpy(X).cuda()
    res = to_np(gw.classify(Xd, torch.from_numpy(s).cuda()))
    slot = np.array(fg["model_of"])[ogw.size_group(s, n_bins=n_bins)]
    for m in range(len(fg["models"])):
        rows = np.nonzero(slot == m)[0]
        if rows.size == 0:
            continue
        Xg, _ = nb.gather(Xd[torch.from_numpy(rows).cuda()], fg["cols"][m:m + 1])
        alone = to_np(nb.score(fg["models"][m], Xg))
        assert (alone["label"] == res["label"][rows]).all()
        assert (alone["margin"] == res["margin"][rows]).all()
        assert (alone["lp"] == res["lp"][rows]).all()


def test_groupwise_routed_path_f32_and_unaligned():
    # F32 histograms, and u8 rows whose pitch is not a multiple of 16, take
    # the route + gather + batched-launch path; same results as the oracle
    n_bins, F, k = 12, 200, 24
    X, y, s = _workload(91, 5000, F, n_bins)
    tr, te = synth.split_per_class(92, y)
    fo = ogw.fit_groups(X[tr], y[tr], s[tr], k, n_bins=n_bins)
    ref = ogw.score_groups(X[te], s[te], fo)
    X32 = torch.from_numpy(X.astype(np.float32)).cuda()
    fg = nb.fit_groupwise(X32[tr], torch.from_numpy(y[tr]).cuda(), torch.from_numpy(s[tr]).cuda(),
                          k, n_bins=n_bins)
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, dtype_code=nb.NB_F32,
                      max_files=len(te))
    res = gw.classify(X32[te], torch.from_numpy(s[te]).cuda())
    torch.cuda.synchronize()
    compare(to_np(res), ref)
    # u8 with a row pitch of F + 4 bytes (rows not 16-byte aligned)
    fg8 = nb.fit_groupwise(torch.from_numpy(X[tr]).cuda(), torch.from_numpy(y[tr]).cuda(),
                           torch.from_numpy(s[tr]).cuda(), k, n_bins=n_bins)
    Xp = torch.zeros((len(te), F + 4), dtype=torch.uint8, device="cuda")
    Xp[:, :F] = torch.from_numpy(X[te]).cuda()
    gw8 = nb.Groupwise(fg8["models"], fg8["cols"], fg8["model_of"], F, max_files=len(te))
    res8 = gw8.classify(Xp[:, :F], torch.from_numpy(s[te]).cuda())
    torch.cuda.synchronize()
    compare(to_np(res8), ref)


def test_groupwise_empty_call():
    n_bins, F, k = 8, 64, 16
    X, y, s = _workload(71, 3000, F, n_bins)
    _, fg = _fit_both(X, y, s, k, nb.NB_SELECT_TOTAL, n_bins)
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=10)
    out = gw.classify(torch.zeros((0, F), dtype=torch.uint8, device="cuda"),
                      torch.zeros(0, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    assert out["label"].numel() == 0


def test_plain_method_with_all_opcodes_in_one_group():
    # k = F and one size group: the group-wise pipeline is plain Naive Bayes
    F = 96
    X, y, _ = _workload(81, 2000, F, 1)
    s = np.full(2000, 1234, np.int64)
    _, fg = _fit_both(X, y, s, F, nb.NB_SELECT_TOTAL, 1)
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=2000)
    res = to_np(gw.classify(torch.from_numpy(X).cuda(), torch.from_numpy(s).cuda()))
    ref = oscore(X.astype(np.float64), mn_fit(X, y, 2))
    compare(res, ref)


@pytest.mark.parametrize("want_lp,recheck", [(False, nb.NB_RECHECK_LABEL), (True, nb.NB_RECHECK_OFF),
                                             (False, nb.NB_RECHECK_LP)])
def test_groupwise_output_and_recheck_options(want_lp, recheck):
    n_bins, F, k = 10, 128, 32
    X, y, s = _workload(101, 5000, F, n_bins)
    tr, te = synth.split_per_class(102, y)
    fo, fg = _fit_both(X[tr], y[tr], s[tr], k, nb.NB_SELECT_TOTAL, n_bins)
    gw = nb.Groupwise(fg["models"], fg["cols"], fg["model_of"], F, max_files=len(te),
                      want_logpost=want_lp, recheck=recheck)
    res = to_np(gw.classify(torch.from_numpy(X[te]).cuda(), torch.from_numpy(s[te]).cuda()))
    ref = ogw.score_groups(X[te], s[te], fo, want_lp=want_lp)
    if recheck == nb.NB_RECHECK_OFF:
        # no recheck: labels may differ only on rows the FP32 bound could not settle
        agree = (res["label"] == ref["label"]).mean()
        assert agree > 0.999
        assert res["n_rechecked"] == 0
    else:
        compare(res, ref, check_lp=want_lp)
