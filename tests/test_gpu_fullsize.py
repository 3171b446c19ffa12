"""Parity at the full size of the two-class benchmark workload, in the launch
configuration the benchmark times: 1,000,000 files x F = 1,024 u16 opcode
counts (Dirichlet(0.1) profiles, lognormal(8.5, 1) totals) stored as u8 rows
plus an overflow list, fit and re-fit on the 2:1 per-class training split
(666,667 files), all 1M files scored by the pipelined scorer with two stages
of 48 rows and two rows per warp pass, log posteriors and FP64 recheck.

The exact class counts are checked against the oracle over the whole training
split (the oracle counts row chunks and the integer sums are added, which is
exact), the FP64 tables against the oracle's finalisation of those counts,
and labels, margins and log posteriors on a seeded sample of 4,096 files
against the oracle's own scoring of them.  Properties that hold at any size
are checked on every file: no row left marked for the recheck, margins
non-negative, the two posteriors of a file summing to one.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import formats
from tests._common import compare, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")

N, F = 1_000_000, 1024


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    nb.build()
    nb.lib()


def _workload():
    # the benchmark's recipe for this configuration, generated on the device
    seed = synth.seed_for(2)
    p = synth.dirichlet_profiles(seed, 2, F, 0.1)
    y = synth.labels_bernoulli(seed + 1, N)
    T = synth.file_totals(seed + 2, N, 8.5, 1.0)
    X16 = synth.count_rows(seed + 3, p, y, T, 65535, out_dtype="uint16", device="cuda",
                           chunk_rows=1 << 16)
    tr, _ = synth.split_per_class(seed + 4, y)
    return X16, y, np.asarray(tr)


def test_benchmark_workload_full_size():
    X16, y, tr = _workload()
    tr_dev = torch.as_tensor(tr, device="cuda")
    X16_tr = X16.view(torch.int16).index_select(0, tr_dev).view(torch.uint16)
    y_tr = torch.as_tensor(y, device="cuda").index_select(0, tr_dev).contiguous()
    low_tr = nb.pack_u8(X16_tr)
    low_all = nb.pack_u8(X16)
    assert low_all.ovf_col.numel() > 0   # the overflow list is exercised

    model = nb.fit(low_tr, y_tr, 2)
    model.set_tile_config(nb.NB_VARIANT_PIPELINED, 2, 48, 2)
    nb.refit(model, low_tr, y_tr)
    res = to_np(nb.score(model, low_all))
    torch.cuda.synchronize()

    # exact counts over the whole training split, chunk by chunk
    y_tr_h = y[tr]
    counts = np.zeros((2, F), np.uint64)
    nc = np.zeros(2, np.uint64)
    step = 65536
    for lo in range(0, len(tr), step):
        hi = min(len(tr), lo + step)
        Xc = X16_tr.view(torch.int16)[lo:hi].cpu().numpy().view(np.uint16)
        m = oracle.mn_fit(Xc, y_tr_h[lo:hi], 2)
        counts += m["counts"]
        nc += m["nc"]
    g_counts, g_nc = model.counts()
    assert (g_counts == counts).all()
    assert (g_nc == nc).all()
    ref_model = oracle.mn_finalize(counts, nc, len(tr))
    lt, _, lpi = model.params()
    assert np.allclose(lt, ref_model["log_theta"], rtol=1e-14, atol=1e-13)
    assert np.allclose(lpi, ref_model["log_pi"], rtol=1e-14, atol=1e-14)

    # labels, margins and log posteriors on a seeded sample, against the oracle
    rows = np.sort(np.random.default_rng(synth.seed_for(2) + 9).choice(N, 4096, replace=False))
    rows_dev = torch.as_tensor(rows, device="cuda")
    Xs = X16.view(torch.int16).index_select(0, rows_dev).cpu().numpy().view(np.uint16)
    ref = oracle.score(Xs, ref_model)
    compare(res, ref, rows=rows)

    # properties of every file
    assert not (res["label"] == 255).any()
    assert (res["label"] <= 1).all()
    assert (res["margin"] >= 0).all()
    s = np.exp(res["lp"].astype(np.float64)).sum(axis=1)
    assert np.abs(s - 1.0).max() < 1e-5


def _sample(n, k, salt):
    return np.sort(np.random.default_rng(synth.seed_for(2) + salt).choice(n, k, replace=False))


def _rows_host(X, rows):
    return X.index_select(0, torch.as_tensor(rows, device=X.device)).cpu().numpy()


def _oracle_counts(Xtr, ytr, C, step=4096, workers=8):
    """Exact class counts of every training row and column, by the oracle.

    The rows go to the host in chunks of ``step``; the oracle counts each
    chunk and the integer counts are added (exact, in any order).  Chunks run
    on a few host threads (the oracle and the copies release the GIL).
    """
    from concurrent.futures import ThreadPoolExecutor

    n, F = Xtr.shape

    def worker(w):   # chunks w, w + workers, ...
        counts = np.zeros((C, F), np.uint64)
        nc = np.zeros(C, np.uint64)
        for lo in range(w * step, n, workers * step):
            hi = min(n, lo + step)
            m = oracle.mn_fit(Xtr[lo:hi].cpu().numpy(), ytr[lo:hi], C)
            counts += m["counts"]
            nc += m["nc"]
        return counts, nc

    counts = np.zeros((C, F), np.uint64)
    nc = np.zeros(C, np.uint64)
    with ThreadPoolExecutor(workers) as ex:
        for c, k in ex.map(worker, range(workers)):
            counts += c
            nc += k
    return counts, nc


def test_many_class_workload_full_size():
    # C = 64 (Zipf 1.1 priors), F = 8,192 u8 counts, N = 2M files: the
    # tensor-core scorer on the whole group; the oracle's exact counts over
    # every training row and column, its scores on sampled rows
    seed = synth.seed_for(4)
    C, Fm, Nm = 64, 8192, 2_000_000
    p = synth.dirichlet_profiles(seed, C, Fm, 0.1)
    y = synth.labels_zipf(seed + 1, Nm, C)
    T = synth.file_totals(seed + 2, Nm, 8.5, 1.0)
    X = torch.empty((Nm, Fm), dtype=torch.uint8, device="cuda")
    synth.count_rows(seed + 3, p, y, T, 255, out_dtype="uint8", device="cuda", out=X,
                     chunk_rows=1 << 15)
    tr, _ = synth.split_per_class(seed + 4, y)
    Xtr = X.index_select(0, torch.as_tensor(tr, device="cuda"))
    ytr = np.asarray(y)[tr]
    model = nb.fit(nb.Features(Xtr, nb.NB_U8), torch.as_tensor(ytr, device="cuda"), C)
    res = to_np(nb.score(model, nb.Features(X, nb.NB_U8)))
    torch.cuda.synchronize()

    g_counts, g_nc = model.counts()
    counts, nc = _oracle_counts(Xtr, ytr, C)
    assert (g_counts == counts).all()
    assert (g_nc == nc).all()
    ref_model = oracle.mn_finalize(counts, nc, len(tr))
    lt, _, lpi = model.params()
    assert np.allclose(lt, ref_model["log_theta"], rtol=1e-14, atol=1e-13)

    rows = _sample(Nm, 2048, 12)
    ref = oracle.score(_rows_host(X, rows), ref_model)
    compare(res, ref, rows=rows)
    assert (res["label"] < C).all()
    s = np.exp(res["lp"].astype(np.float64)).sum(axis=1)
    assert np.abs(s - 1.0).max() < 1e-5

    # the same rows stored BF16 (exact below 256) and FP8 E4M3 (rounded, row
    # scale 2^0), scored on the tensor cores as the benchmark times them
    host = _rows_host(X, rows)
    for tdt, code in ((torch.bfloat16, nb.NB_BF16), (torch.float8_e4m3fn, nb.NB_FP8E4M3)):
        Xs = torch.empty((Nm, Fm), dtype=tdt, device="cuda")
        for r0 in range(0, Nm, 1 << 17):
            Xs[r0:r0 + (1 << 17)] = X[r0:r0 + (1 << 17)].to(torch.float32).to(tdt)
        f = nb.Features(Xs.view(torch.uint8) if code == nb.NB_FP8E4M3 else Xs, code)
        assert nb.score_path(model, f) == nb.NB_PATH_TENSOR
        r = to_np(nb.score(model, f))
        torch.cuda.synchronize()
        if code == nb.NB_BF16:
            vals = host.astype(np.float64)
        else:
            codes, e = formats.pack_e4m3(host)
            assert (e == 0).all()
            assert (_rows_host(Xs.view(torch.uint8), rows) == codes).all()
            vals = formats.unpack_e4m3(codes, e)
        compare(r, oracle.score(vals, ref_model), rows=rows)
        assert (r["label"] < C).all()
        del Xs, f
        torch.cuda.empty_cache()


def test_feature_sweep_widest_point_full_size():
    # F = 16,384, N = 1M u8 counts (Dirichlet(0.05) profiles, 30% shared),
    # fit on the first third; u8 and FP8 E4M3 rows (per-row exponent) scored
    # with log posteriors: the oracle on sampled rows
    seed = synth.seed_for(3)
    Fs = 16384
    Ns = 1_000_000
    p = synth.dirichlet_profiles(seed + Fs, 2, Fs, 0.05, shared_frac=0.3)
    y = synth.labels_bernoulli(seed + Fs + 1, Ns)
    T = synth.file_totals(seed + Fs + 2, Ns, 8.5, 1.0)
    X = torch.empty((Ns, Fs), dtype=torch.uint8, device="cuda")
    synth.count_rows(seed + Fs + 3, p, y, T, 255, out_dtype="uint8", device="cuda", out=X,
                     chunk_rows=max(1024, (1 << 27) // Fs))
    ntr = Ns // 3
    y = np.asarray(y)
    model = nb.fit(nb.Features(X[:ntr], nb.NB_U8), torch.as_tensor(y[:ntr], device="cuda"), 2)
    res = to_np(nb.score(model, nb.Features(X, nb.NB_U8)))

    g_counts, g_nc = model.counts()
    counts, nc = _oracle_counts(X[:ntr], y[:ntr], 2)
    assert (g_counts == counts).all()
    assert (g_nc == nc).all()
    ref_model = oracle.mn_finalize(counts, nc, ntr)

    rows = _sample(Ns, 2048, 22)
    Xs = _rows_host(X, rows)
    compare(res, oracle.score(Xs, ref_model), rows=rows)

    # FP8 rows, packed on the device in row chunks
    codes = torch.empty((Ns, Fs), dtype=torch.uint8, device="cuda")
    rexp = torch.empty(Ns, dtype=torch.int8, device="cuda")
    step = 1 << 15
    for lo in range(0, Ns, step):
        f = nb.pack_fp8(X[lo:lo + step].to(torch.float32))
        codes[lo:lo + step].copy_(f.data)
        rexp[lo:lo + step].copy_(f.row_exp)
    f8 = nb.Features(codes, nb.NB_FP8E4M3, row_exp=rexp)
    c8, e8 = _rows_host(codes, rows), _rows_host(rexp, rows)
    ref_codes, ref_e = formats.pack_e4m3(Xs)
    assert (c8 == ref_codes).all() and (e8 == ref_e).all()
    ref8 = oracle.score(formats.unpack_e4m3(ref_codes, ref_e), ref_model)
    # the default shape and the register-streaming kernel: exact integer
    # counts, so labels and log posteriors both meet the tolerance, and the two
    # kernels give the same bits
    outs = []
    for cfg in [(nb.NB_VARIANT_AUTO, 0, 0, 0), (nb.NB_VARIANT_REGISTER, 0, 0, 0)]:
        model.set_tile_config(*cfg)
        res8 = to_np(nb.score(model, f8, recheck=nb.NB_RECHECK_LP))
        torch.cuda.synchronize()
        compare(res8, ref8, rows=rows)
        assert not (res8["label"] == 255).any()
        outs.append(res8)
    assert (outs[0]["label"] == outs[1]["label"]).all()
    assert (outs[0]["margin"].view(np.uint32) == outs[1]["margin"].view(np.uint32)).all()
