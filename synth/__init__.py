"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and
the benchmark.

The paper's data (Malicia malware and Windows benign executables reduced to
opcode occurrence counts, Sec. 3) is not available, so these generators give
inputs with its structure: non-negative per-file opcode-count vectors, two
classes (benign = 0, malware = 1) or many families, files arriving in groups.
This module draws random numbers only; it holds none of the Naive Bayes
arithmetic.  Everything is a pure function of its seed.

Recipes (sizes are parameters; the defaults are the workloads' own):

* ``gaussian_workload`` -- C = 2, F = 64; per-class means ~ U(0, 10) and
  standard deviations ~ U(0.5, 3); x ~ N(mu_c, sd_c^2) drawn in FP64, stored
  FP32; 1,000 fit and 5,000 scored files per class.
* ``dirichlet_profiles`` -- per-class feature distributions p_c ~
  Dirichlet(conc * 1_F); optionally a shared block: a seeded fraction of the
  features carries weight ``shared_weight`` with one profile common to all
  classes, the rest a per-class profile (the "30 % shared features" sweep).
* ``count_rows`` -- file totals T_i = round(lognormal(mu, sigma)) and counts
  x_ij ~ Poisson(T_i * p_{y_i, j}), clipped to the storage maximum.  (Poisson
  splitting: conditioned on their sum, independent Poisson counts are exactly
  multinomial, so this is the multinomial event model with a Poisson total.)
  Draws run through ``torch.poisson`` with a seeded generator on the chosen
  device, in row chunks, so the 1M-64M-row workloads build in seconds.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1905_13746


def seed_for(config_index: int) -> int:
    """Fixed seed of workload number ``config_index`` (1-based)."""
    return SEED_BASE + int(config_index)


# ----------------------------------------------------------------------------
# Gaussian workload
# ----------------------------------------------------------------------------
def gaussian_workload(seed, F=64, C=2, n_fit_per_class=1000,
                      n_score_per_class=5000, spread=10.0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(0.0, spread, size=(C, F))
    sd = rng.uniform(0.5, 3.0, size=(C, F))

    def draw(n_per):
        y = np.repeat(np.arange(C, dtype=np.int32), n_per)
        y = y[rng.permutation(y.shape[0])]
        X = rng.normal(mu[y], sd[y]).astype(np.float32)
        return X, y

    X_fit, y_fit = draw(n_fit_per_class)
    X_score, y_score = draw(n_score_per_class)
    return {"X_fit": X_fit, "y_fit": y_fit, "X_score": X_score,
            "y_score": y_score, "mu": mu, "sd": sd,
            "log_prior": np.log(np.full(C, 1.0 / C))}


# ----------------------------------------------------------------------------
# Count workloads
# ----------------------------------------------------------------------------
def dirichlet_profiles(seed, C, F, conc, shared_frac=0.0, shared_weight=0.3):
    """C x F float64 rows summing to 1."""
    rng = np.random.default_rng(seed)
    if shared_frac <= 0.0:
        return rng.dirichlet(np.full(F, conc), size=C)
    k = max(1, int(round(shared_frac * F)))
    shared_idx = np.sort(rng.permutation(F)[:k])
    own_idx = np.setdiff1d(np.arange(F), shared_idx)
    q_s = rng.dirichlet(np.full(k, conc))
    p = np.zeros((C, F))
    for c in range(C):
        p[c, shared_idx] = shared_weight * q_s
        p[c, own_idx] = (1.0 - shared_weight) * rng.dirichlet(np.full(F - k, conc))
    return p


def labels_bernoulli(seed, n, p_malware=0.5):
    rng = np.random.default_rng(seed)
    return (rng.random(n) < p_malware).astype(np.int32)


def labels_zipf(seed, n, C, s=1.1):
    """Class c drawn with probability proportional to (c + 1)^-s."""
    rng = np.random.default_rng(seed)
    w = (np.arange(C) + 1.0) ** (-s)
    return rng.choice(C, size=n, p=w / w.sum()).astype(np.int32)


def file_totals(seed, n, mu=8.5, sigma=1.0):
    rng = np.random.default_rng(seed)
    return np.rint(rng.lognormal(mu, sigma, size=n))


def count_rows(seed, p, y, totals, clip, out_dtype="uint16", device="cpu",
               chunk_rows=1 << 16, out=None):
    """Counts x_ij ~ Poisson(T_i p_{y_i j}) clipped to ``clip`` (torch tensor).

    ``out`` may be a preallocated (n x F) torch tensor of ``out_dtype`` (any
    device); rows are produced in chunks of ``chunk_rows``.
    """
    import torch

    n = int(y.shape[0])
    F = int(p.shape[1])
    tdt = {"uint16": torch.int32, "uint8": torch.uint8, "float32": torch.float32}
    store = {"uint16": torch.uint16 if hasattr(torch, "uint16") else torch.int32,
             "uint8": torch.uint8, "float32": torch.float32}[out_dtype]
    if out is None:
        out = torch.empty((n, F), dtype=store, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    p_dev = torch.as_tensor(p, dtype=torch.float32, device=device)
    y_dev = torch.as_tensor(np.asarray(y, np.int64), device=device)
    t_dev = torch.as_tensor(np.asarray(totals, np.float32), device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        rates = t_dev[r0:r1, None] * p_dev[y_dev[r0:r1]]
        x = torch.poisson(rates, generator=g).clamp_(max=float(clip))
        if out_dtype == "float32":
            out[r0:r1] = x.to(out.device)
        else:
            out[r0:r1] = x.to(torch.int32).to(store).to(out.device)
        del rates, x
    _ = tdt
    return out


def split_per_class(seed, y, train_frac=2.0 / 3.0):
    """Per-class random split (the paper's 2:1 split, done class by class).

    Returns (train_idx, test_idx), each sorted ascending.
    """
    rng = np.random.default_rng(seed)
    train, test = [], []
    for c in np.unique(y):
        idx = np.nonzero(y == c)[0]
        idx = idx[rng.permutation(idx.shape[0])]
        k = int(math.ceil(train_frac * idx.shape[0]))
        train.append(idx[:k])
        test.append(idx[k:])
    return np.sort(np.concatenate(train)), np.sort(np.concatenate(test))


# ----------------------------------------------------------------------------
# Serving workload: groups of files and their arrivals
# ----------------------------------------------------------------------------
def group_sizes(seed, n_groups, median=500, sigma=1.49, lo=1, hi=50_000):
    rng = np.random.default_rng(seed)
    s = np.rint(rng.lognormal(math.log(median), sigma, size=n_groups))
    return np.clip(s, lo, hi).astype(np.int64)


def poisson_arrivals(seed, n, rate_per_s):
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def model_choice(seed, n, n_models=2):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n_models, size=n).astype(np.int32)


# ----------------------------------------------------------------------------
# Group-wise workload: files with sizes, grouped opcode profiles
# ----------------------------------------------------------------------------
def groupwise_workload(seed, n, F, n_bins=100, bin_bytes=5 * 1024, C=2, conc=0.1, mix=0.5,
                       bytes_per_opcode=16, p_malware=0.827, bin_median=12.0,
                       bin_sigma=1.0, clip=255, out_dtype="uint8", device="cpu"):
    """Files of Sec. 3's kind: a size window, a class, an opcode histogram.

    * window w_i of ``bin_bytes`` drawn with weights ~ lognormal in the window
      index (median ``bin_median``, log-sd ``bin_sigma``): most files are small,
      as the paper's population below 500 KB;  size_i = w_i * bin_bytes +
      U[0, bin_bytes);
    * class: malware with probability ``p_malware`` (11,305 of 13,665 files in
      the paper's data set);
    * opcode profile of (window, class): ``mix`` x a class profile common to
      all windows + (1 - mix) x a window-specific one, each Dirichlet(conc);
    * opcode total T_i = max(1, size_i // bytes_per_opcode), counts
      x_ij ~ Poisson(T_i p_j) clipped to ``clip`` (u8: 255).
    Returns (X torch tensor n x F, y int32 numpy, sizes int64 numpy).
    """
    rng = np.random.default_rng(seed)
    idx = np.arange(n_bins) + 0.5
    w = np.exp(-0.5 * ((np.log(idx) - math.log(bin_median)) / bin_sigma) ** 2) / idx
    win = rng.choice(n_bins, size=n, p=w / w.sum())
    sizes = (win * bin_bytes + rng.integers(0, bin_bytes, size=n)).astype(np.int64)
    y = (rng.random(n) < p_malware).astype(np.int32)
    base = dirichlet_profiles(seed + 1, C, F, conc)
    local = np.random.default_rng(seed + 2).dirichlet(np.full(F, conc), size=(n_bins, C))
    prof = (mix * base[None, :, :] + (1.0 - mix) * local).reshape(n_bins * C, F)
    T = np.maximum(1, sizes // bytes_per_opcode)
    X = count_rows(seed + 3, prof, win * C + y, T, clip, out_dtype=out_dtype, device=device)
    return X, y, sizes
