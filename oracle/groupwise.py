"""Group-wise pipeline of the paper (Sec. 3 and Sec. 4) -- oracle, test
infrastructure only (the same import rule as the rest of ``oracle``).

Plain Python / numpy, exact where the method is exact:

* ``size_group`` -- Sec. 3 partitions the files below 500 KB into 100 groups
  of 5 KB each.  Reading: group g = floor(size / 5120) (a KB is 1024 bytes),
  and a file of 500 KB or more, outside the paper's population, joins the
  last group instead of being dropped.
* ``group_models`` -- Sec. 4 trains one model per group, except for groups
  with fewer than six files of either class, whose files are classified with
  the next group's model.  Reading: a group is trained when each class has at
  least ``min_files`` training files; an untrained group takes the first
  trained group above it, and when there is none (the last groups), the
  nearest trained group below it.
* ``select_features`` -- Sec. 3 keeps, per group, the k opcodes whose
  normalised occurrence differs most between malware and benign files.  The
  normalisation itself is only cited, not stated.  Reading: f_cj = N_cj / D_c
  with N_cj the group's class-c total count of opcode j and D_c either the
  class's total opcode count (``norm="total"``, f_c is the class's opcode
  distribution) or its number of files (``norm="files"``, f_c is the mean
  count per file); a class with D_c = 0 has f_c = 0.  Rank j by |f_1j - f_0j|
  (exact rational arithmetic), larger first, ties to the lower opcode index;
  the selection is the first k of that ranking, in rank order.
* ``gather`` -- the selected columns of a full histogram, in selection order.
* ``fit_groups`` / ``score_groups`` -- the whole method: per trained group,
  rank on the group's training files, fit Naive Bayes (``oracle.mn_fit``) on
  the selected columns; a scored file goes to its group's model (or the
  fallback), is reduced to that model's columns and scored (``oracle.score``).

Nothing here is blocked, fused or reordered beyond these definitions.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from . import mn_fit, score

BIN_BYTES = 5 * 1024     # Sec. 3: groups of 5 KB
N_BINS = 100             # Sec. 3: 100 groups (files below 500 KB)
MIN_FILES = 6            # Sec. 4: fewer than six files of a class -> untrained

NORMS = ("total", "files")


def size_group(sizes, bin_bytes=BIN_BYTES, n_bins=N_BINS):
    """Group index of each file size in bytes (Sec. 3), as int64."""
    out = []
    for s in np.asarray(sizes).tolist():
        s = int(s)
        if s < 0:
            raise ValueError("file sizes are non-negative")
        out.append(min(s // bin_bytes, n_bins - 1))
    return np.array(out, dtype=np.int64)


def group_class_counts(groups, y, n_bins=N_BINS, C=2):
    """Training files per (group, class)."""
    cnt = np.zeros((n_bins, C), np.int64)
    for g, c in zip(np.asarray(groups).tolist(), np.asarray(y).tolist()):
        cnt[g, c] += 1
    return cnt


def group_models(class_counts, min_files=MIN_FILES):
    """Model group of every group (Sec. 4 small-group rule).

    class_counts: (n_bins, C) training files per group and class.  Returns an
    int64 array m with m[g] = g for a trained group, else the first trained
    group above g, else the nearest trained group below g.  Raises ValueError
    when no group is trained.
    """
    cc = np.asarray(class_counts)
    n_bins = cc.shape[0]
    trained = [bool(min(cc[g].tolist()) >= min_files) for g in range(n_bins)]
    if not any(trained):
        raise ValueError("no group has enough training files of every class")
    out = []
    for g in range(n_bins):
        m = None
        for h in range(g, n_bins):          # this group, then upward
            if trained[h]:
                m = h
                break
        if m is None:
            for h in range(g - 1, -1, -1):  # none above: downward
                if trained[h]:
                    m = h
                    break
        out.append(m)
    return np.array(out, dtype=np.int64)


def feature_scores(counts, nfiles, norm="total"):
    """Exact |f_1j - f_0j| for a two-class group, as Fractions.

    counts: (2, F) integer counts N_cj; nfiles: (2,) files per class.
    """
    if norm not in NORMS:
        raise ValueError(f"norm must be one of {NORMS}")
    N = [[int(v) for v in row] for row in np.asarray(counts, dtype=np.uint64).tolist()]
    if len(N) != 2:
        raise ValueError("feature selection compares two classes")
    if norm == "total":
        D = [sum(N[0]), sum(N[1])]
    else:
        D = [int(v) for v in np.asarray(nfiles).tolist()]
    F = len(N[0])
    f = [[Fraction(N[c][j], D[c]) if D[c] > 0 else Fraction(0) for j in range(F)]
         for c in range(2)]
    return [abs(f[1][j] - f[0][j]) for j in range(F)]


def select_features(counts, nfiles, k, norm="total"):
    """The k top-ranked opcodes of a group, in rank order (int32)."""
    sc = feature_scores(counts, nfiles, norm)
    F = len(sc)
    if not 1 <= k <= F:
        raise ValueError("need 1 <= k <= F")
    order = sorted(range(F), key=lambda j: (-sc[j], j))
    return np.array(order[:k], dtype=np.int32)


def gather(X, cols):
    """Columns ``cols`` of each row of X, in that order."""
    X = np.asarray(X)
    return X[:, np.asarray(cols, dtype=np.int64)]


def fit_groups(X, y, sizes, k, norm="total", alpha=1.0, bin_bytes=BIN_BYTES,
               n_bins=N_BINS, min_files=MIN_FILES):
    """Train the per-group models of the method on full histograms X (n x F).

    Returns {"model_of": group -> model group, "cols": {g: selection},
    "models": {g: oracle model on the selected columns}} for trained g.
    """
    X = np.asarray(X)
    y = np.asarray(y)
    g = size_group(sizes, bin_bytes, n_bins)
    cc = group_class_counts(g, y, n_bins, 2)
    model_of = group_models(cc, min_files)
    cols, models = {}, {}
    for b in sorted(set(model_of.tolist())):
        rows = np.nonzero(g == b)[0]
        Xb, yb = X[rows], y[rows]
        counts = np.zeros((2, X.shape[1]), np.uint64)
        for c in range(2):
            counts[c] = X[rows[yb == c]].astype(np.uint64).sum(axis=0)
        cols[b] = select_features(counts, cc[b], k, norm)
        models[b] = mn_fit(gather(Xb, cols[b]), yb, 2, alpha)
    return {"model_of": model_of, "cols": cols, "models": models,
            "bin_bytes": bin_bytes, "n_bins": n_bins}


def score_groups(X, sizes, fitted, want_lp=True):
    """Classify files with the group-wise models: per file label, margin, lp
    (in the files' own order) and the model group used."""
    X = np.asarray(X)
    g = size_group(sizes, fitted["bin_bytes"], fitted["n_bins"])
    m = fitted["model_of"][g]
    n = X.shape[0]
    label = np.zeros(n, np.uint8)
    margin = np.zeros(n, np.float64)
    lp = np.zeros((n, 2), np.float64)
    for b in sorted(set(m.tolist())):
        rows = np.nonzero(m == b)[0]
        r = score(gather(X[rows], fitted["cols"][b]), fitted["models"][b], want_lp=want_lp)
        label[rows] = r["label"]
        margin[rows] = r["margin"]
        if want_lp:
            lp[rows] = r["lp"]
    return {"label": label, "margin": margin, "lp": lp if want_lp else None, "model": m}
