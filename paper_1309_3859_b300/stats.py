"""Host-side statistics over per-measurement records.

The multilevel estimators of the paper (Section II.C) are averages over
independent measurements; their errors follow from the jackknife over
measurements (Section III.C, "we use the jackknife method").
"""

from __future__ import annotations

import numpy as np


def jackknife(samples: np.ndarray, fn=None, axis: int = 0):
    """Jackknife mean and standard error of ``fn`` over leave-one-out means.

    ``samples`` holds one row per measurement along ``axis``.  ``fn`` maps a
    mean over rows to the estimate (identity when None), so ratios of means
    such as <P+P O> / <P+P> get their correlated error.
    """
    x = np.moveaxis(np.asarray(samples), axis, 0)
    n = x.shape[0]
    if fn is None:
        fn = lambda m: m  # noqa: E731
    full = fn(x.mean(axis=0))
    if n < 2:
        return full, np.full_like(np.asarray(full, dtype=float), np.inf)
    tot = x.sum(axis=0)
    loo = np.stack([fn((tot - x[i]) / (n - 1)) for i in range(n)])
    err = np.sqrt((n - 1) / n * ((loo - loo.mean(axis=0)) ** 2).sum(axis=0))
    return full, err


def binned(samples: np.ndarray, bin_size: int) -> np.ndarray:
    """Means over consecutive bins of ``bin_size`` rows (drops a ragged tail)."""
    x = np.asarray(samples)
    n = (x.shape[0] // bin_size) * bin_size
    return x[:n].reshape((n // bin_size, bin_size) + x.shape[1:]).mean(axis=1)
