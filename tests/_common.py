"""Helpers shared by the GPU parity tests: seeded inputs in each storage format
with their exact (dequantised) values for the oracle, and the comparisons.

The oracle-side values always come from ``synth`` (the generator) and
``oracle.formats`` (format definitions), never from the CUDA library.
"""
import numpy as np
import torch

import oracle
import synth
from oracle import formats

LP_TOL = 1e-5          # |lp - lp_ref| <= LP_TOL * max(1, |lp_ref|)


def count_matrix(seed, n, F, C=2, conc=0.1, clip=65535, mu=8.5, sigma=1.0, labels=None,
                 p=None):
    """(X u16/u8 numpy, y int32) with Poisson-split multinomial rows."""
    if p is None:
        p = synth.dirichlet_profiles(seed, C, F, conc)
    y = synth.labels_bernoulli(seed + 1, n) if (labels is None and C == 2) else labels
    if y is None:
        y = synth.labels_zipf(seed + 1, n, C)
    T = synth.file_totals(seed + 2, n, mu, sigma)
    out_dtype = "uint8" if clip <= 255 else "uint16"
    X = synth.count_rows(seed + 3, p, y, T, clip, out_dtype=out_dtype, device="cpu")
    Xn = X.view(torch.int16).numpy().view(np.uint16) if out_dtype == "uint16" else X.numpy()
    return Xn.copy(), np.asarray(y, np.int32), p


def stored(X, fmt):
    """Device Features of storage ``fmt`` for counts X (numpy) + exact values (f64).

    The packed forms are built on the host by ``oracle.formats`` (the format
    definitions), so the GPU scorer and the oracle read the same values.
    """
    import paper_1905_13746_gb300 as nb
    X = np.asarray(X)
    n, F = X.shape
    dev = "cuda"
    if fmt == "u16":
        t = torch.from_numpy(X.astype(np.uint16).view(np.int16)).to(dev).view(torch.uint16)
        return nb.Features(t, nb.NB_U16), X.astype(np.float64)
    if fmt == "f32":
        return nb.Features(torch.from_numpy(X.astype(np.float32)).to(dev), nb.NB_F32), \
            X.astype(np.float64)
    if fmt == "u8ovf":
        plane, ptr, col, add = formats.pack_u8_overflow(X)
        ldp = (F + 15) // 16 * 16
        P = np.zeros((n, ldp), np.uint8)
        P[:, :F] = plane
        tp = torch.from_numpy(P).to(dev)[:, :F]
        # side arrays are never empty buffers (the C ABI wants non-NULL pointers)
        colp = np.zeros(max(1, col.size), np.uint16)
        addp = np.zeros(max(1, add.size), np.uint16)
        colp[:col.size], addp[:add.size] = col, add
        f = nb.Features(tp, nb.NB_U8,
                        torch.from_numpy(ptr).to(dev),
                        torch.from_numpy(colp.view(np.int16)).to(dev),
                        torch.from_numpy(addp.view(np.int16)).to(dev))
        return f, formats.unpack_u8_overflow(plane, ptr, col, add) if n * F <= 4_000_000 \
            else X.astype(np.float64)
    if fmt == "u8":
        Xc = np.minimum(X, 255).astype(np.uint8)
        ldp = (F + 15) // 16 * 16
        P = np.zeros((n, ldp), np.uint8)
        P[:, :F] = Xc
        return nb.Features(torch.from_numpy(P).to(dev)[:, :F], nb.NB_U8), Xc.astype(np.float64)
    if fmt == "bf16":
        bits = formats.bf16_bits(X)
        ldp = (F + 7) // 8 * 8
        B = np.zeros((n, ldp), np.uint16)
        B[:, :F] = bits
        t = torch.from_numpy(B.view(np.int16)).to(dev).view(torch.bfloat16)[:, :F]
        return nb.Features(t, nb.NB_BF16), formats.bf16_decode(bits)
    if fmt == "fp8":
        codes, e = formats.pack_e4m3(X)
        ldp = (F + 15) // 16 * 16
        B = np.zeros((n, ldp), np.uint8)
        B[:, :F] = codes
        f = nb.Features(torch.from_numpy(B).to(dev)[:, :F], nb.NB_FP8E4M3,
                        row_exp=torch.from_numpy(e).to(dev))
        return f, formats.unpack_e4m3(codes, e)
    raise ValueError(fmt)


def to_np(res):
    out = {"label": res["label"].cpu().numpy(), "margin": res["margin"].cpu().numpy()}
    out["lp"] = res["logpost"].cpu().numpy() if res.get("logpost") is not None else None
    out["n_rechecked"] = int(res["n_rechecked"].cpu().item()) if "n_rechecked" in res else None
    return out


def compare(got, ref, lp_tol=LP_TOL, check_lp=True, rows=None):
    """Labels bit-exact; lp within lp_tol*max(1,|lp|); margin within the same."""
    lab, mar = got["label"], got["margin"].astype(np.float64)
    rl, rm = ref["label"], ref["margin"]
    if rows is not None:
        lab, mar = lab[rows], mar[rows]
    bad = np.nonzero(lab != rl)[0]
    assert bad.size == 0, f"{bad.size} label mismatches, first rows {bad[:10]} " \
        f"(gpu {lab[bad[:5]]}, ref {rl[bad[:5]]}, ref margin {rm[bad[:5]]})"
    merr = np.abs(mar - rm) / np.maximum(1.0, np.abs(rm))
    stats = {"margin_err": float(merr.max()) if merr.size else 0.0}
    if check_lp:
        assert (merr <= lp_tol).all(), f"margin rel err {merr.max():.3e}"
    if ref.get("lp") is not None and got.get("lp") is not None:
        lp = got["lp"].astype(np.float64)
        if rows is not None:
            lp = lp[rows]
        err = np.abs(lp - ref["lp"]) / np.maximum(1.0, np.abs(ref["lp"]))
        stats["lp_err"] = float(err.max()) if err.size else 0.0
        if check_lp:
            assert (err <= lp_tol).all(), \
                f"lp rel err {err.max():.3e} at row {np.unravel_index(err.argmax(), err.shape)}"
    return stats


def oracle_mn(Xfit, yfit, C, Xscore, alpha=1.0, log_prior=None):
    m = oracle.mn_fit(Xfit, yfit, C, alpha=alpha, log_prior=log_prior)
    return m, oracle.score(Xscore, m)
