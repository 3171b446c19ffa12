"""Segmented batches (one persistent launch per kernel family, optionally
replayed from a captured CUDA graph) against single-group scoring and the
oracle: each group's labels, margins and log posteriors must be the same bits
as when the group is scored alone (Sec. 4 posterior and decision rule, the
paper's groups of Sec. 3)."""
import numpy as np
import pytest
import torch

import synth
from tests._common import compare, count_matrix, oracle_mn, stored, to_np

pytestmark = pytest.mark.gpu

nb = pytest.importorskip("paper_1905_13746_gb300")


def _clip(fmt):
    # counts of the compact formats stay where they are exact (u8) or where the
    # tensor-core scorer takes every row (BF16, FP8 with row scale 2^0)
    return 255 if fmt in ("u8", "bf16", "fp8") else 65535


def _models(F, fmt, seed, Cs):
    out = []
    for i, C in enumerate(Cs):
        X, y, _ = count_matrix(seed + 17 * i, 3000, F, C=C, clip=_clip(fmt))
        f, vals = stored(X, fmt)
        out.append((nb.fit(f, torch.from_numpy(y).cuda(), C), vals, y))
    return out


def _groups(F, fmt, seed, sizes, n_models, Cs):
    groups = []
    for k, n in enumerate(sizes):
        slot = k % n_models
        X, _, _ = count_matrix(seed + 101 * k, max(n, 1), F, C=Cs[slot], clip=_clip(fmt))
        X = X[:n]
        f, v = stored(X, fmt)
        groups.append((slot, f, v))
    return groups


def _check_against_single(models, batch, groups, single_outs):
    outs = [batch.outputs(slot, f.n) for slot, f, _ in groups]
    nre = torch.zeros(1, dtype=torch.int64, device="cuda")
    batch.score([(slot, f, o) for (slot, f, _), o in zip(groups, outs)], n_rechecked=nre)
    torch.cuda.synchronize()
    for (slot, f, v), o, ref in zip(groups, outs, single_outs):
        got = to_np(dict(o, n_rechecked=torch.zeros(1)))
        assert (got["label"] == ref["label"]).all()
        assert (got["margin"].view(np.uint32) == ref["margin"].view(np.uint32)).all()
        assert (got["lp"].view(np.uint32) == ref["lp"].view(np.uint32)).all()
    return int(nre.item())


@pytest.mark.parametrize("fmt", ["u8ovf", "u8", "f32", "bf16", "fp8"])
def test_batch_equals_single_groups_and_oracle(fmt):
    F = 1024 if fmt != "u8" else 2048
    # two-class models batch U8 or F32 rows; BF16 and FP8 batches hold
    # many-class models, whose groups take the tensor-core kernel
    Cs = {"f32": [2, 3], "bf16": [3, 16], "fp8": [16, 5]}.get(fmt, [2, 2, 3])
    mods = _models(F, fmt, 5, Cs)
    sizes = [1, 17, 530, 5003, 0, 64, 1000, 2, 31, 33, 12000, 7]
    groups = _groups(F, fmt, 900, sizes, len(mods), Cs)
    dtype = groups[0][1].dtype_code
    single = []
    for slot, f, v in groups:
        r = to_np(nb.score(mods[slot][0], f)) if f.n else None
        if f.n:
            _, ref = oracle_mn(mods[slot][1], mods[slot][2], Cs[slot], v)
            compare(r, ref, check_lp=Cs[slot] == 2)
        single.append(r if r is not None else {"label": np.zeros(0, np.uint8),
                                               "margin": np.zeros(0, np.float32),
                                               "lp": np.zeros((0, Cs[slot]), np.float32)})
    batch = nb.Batch([m for m, _, _ in mods], dtype, max(f.ld for _, f, _ in groups), 64)
    _check_against_single(mods, batch, groups, single)
    # graph replay, twice, with a different mix the second time
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        batch.capture(st)
        _check_against_single(mods, batch, groups, single)
        perm = list(reversed(range(len(groups))))
        _check_against_single(mods, batch, [groups[i] for i in perm], [single[i] for i in perm])
    st.synchronize()


def test_batch_rejects_bad_groups():
    mods = _models(256, "u8", 3, [2])
    # two-class models batch u8 or f32 rows only
    for dt in (nb.NB_FP8E4M3, nb.NB_BF16, nb.NB_U16):
        with pytest.raises(nb.NbError):
            nb.Batch([mods[0][0]], dt, 256, 4)
    f, _ = stored(np.zeros((10, 256), np.int64), "u8")
    batch = nb.Batch([mods[0][0]], nb.NB_U8, 256, 4)
    out = batch.outputs(0, 10)
    with pytest.raises(nb.NbError):
        batch.score([(1, f, out)])            # no such model slot
    with pytest.raises(nb.NbError):
        batch.score([(0, f, out)] * 5)        # more groups than max_groups
