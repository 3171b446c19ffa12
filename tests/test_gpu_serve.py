"""The serving loop (continuous batching of arriving groups): every group's
result from the mixed stream must be the same bits as scoring that group
alone; waits time out on the host; oversize groups are refused."""
import numpy as np
import pytest
import torch

from tests._common import count_matrix, stored, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")

F = 512


def _models():
    out = []
    for i, C in enumerate([2, 16]):
        X, y, _ = count_matrix(40 + i, 4000, F, C=C, clip=255)
        f, _ = stored(X, "u8")
        out.append(nb.fit(f, torch.from_numpy(y).cuda(), C))
    return out


def test_stream_results_equal_single_group_scoring():
    models = _models()
    server = nb.Server(models, nb.NB_U8, mem_budget=64 << 20, max_slots=16)
    rng = np.random.default_rng(3)
    jobs = []
    for k in range(60):
        mid = int(k % 2)
        n = int(np.clip(rng.lognormal(np.log(300), 1.2), 1, 5000))
        X, _, _ = count_matrix(1000 + k, n, F, C=models[mid].C, clip=255)
        Xt = torch.from_numpy(X.astype(np.uint8))
        on_device = k % 3 == 0
        Xs = Xt.cuda() if on_device else Xt.pin_memory()
        # outputs: device memory, pinned host memory, or pageable host memory
        out = server.outputs(mid, n, device="cuda" if on_device else "cpu", pin=k % 4 != 1)
        jobs.append((mid, Xt, out, server.submit(mid, Xs, out)))
    for mid, Xt, out, t in jobs:
        server.wait(t, timeout_us=30_000_000)
    torch.cuda.synchronize()
    for mid, Xt, out, t in jobs:
        ref = to_np(nb.score(models[mid], Xt.cuda()))
        got = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
        assert (got["label"] == ref["label"]).all()
        assert (got["margin"].view(np.uint32) == ref["margin"].view(np.uint32)).all()
        assert (got["logpost"].view(np.uint32) == ref["lp"].view(np.uint32)).all()
    st = server.stats()
    assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"] and st["files_per_s"] > 0
    server.close()


def test_wait_times_out_and_oversize_is_refused():
    models = _models()
    server = nb.Server(models, nb.NB_U8, mem_budget=16 << 20, max_slots=4)
    X = torch.zeros((20000, F), dtype=torch.uint8).pin_memory()
    out = server.outputs(1, 20000)
    t = server.submit(1, X, out)
    with pytest.raises(nb.NbError) as ei:
        server.wait(t, timeout_us=0)
    assert ei.value.status == nb.NB_ETIMEOUT
    server.wait(t, timeout_us=30_000_000)
    assert (out["label"].numpy() != 255).all()
    big = torch.zeros((100_000, F), dtype=torch.uint8).pin_memory()   # > 16 MiB staged
    with pytest.raises(nb.NbError) as ei:
        server.submit(0, big, server.outputs(0, 100_000))
    assert ei.value.status == nb.NB_EBUSY
    with pytest.raises(nb.NbError):
        server.wait(12345)
    server.close()


def test_burst_submission_with_scheduled_arrivals():
    models = _models()
    server = nb.Server(models, nb.NB_U8, mem_budget=64 << 20, max_slots=8)
    rng = np.random.default_rng(5)
    items, refs = [], []
    for k in range(20):
        mid = int(rng.integers(0, 2))
        n = int(rng.integers(1, 3000))
        X, _, _ = count_matrix(2000 + k, n, F, C=models[mid].C, clip=255)
        Xt = torch.from_numpy(X.astype(np.uint8))
        items.append((mid, Xt.pin_memory(), server.outputs(mid, n)))
        refs.append(to_np(nb.score(models[mid], Xt.cuda())))
    # every group "arrived" 50 ms before the burst was handed over
    t0 = nb.Server.clock_us() - 50_000.0
    tickets = server.submit_many(items, arrival_us=[t0] * len(items))
    assert len(set(tickets)) == len(items)
    for t in tickets:
        server.wait(t, timeout_us=30_000_000)
    for (mid, _, out), ref in zip(items, refs):
        assert (out["label"].numpy() == ref["label"]).all()
        assert (out["margin"].numpy().view(np.uint32) == ref["margin"].view(np.uint32)).all()
    st = server.stats()
    assert st["p50_us"] >= 50_000.0
    with pytest.raises(nb.NbError):          # a bad model id stops the burst there
        server.submit_many([items[0][:1] + items[0][1:], (7,) + items[0][1:]])
    server.close()
