"""Helpers shared by the parity tests and the benchmark: comparison of a GPU
periodogram against the oracle on a set of bins, with the tolerance rules.

Tolerance (readings stated in the design notes):
  * strict bins (oracle relative pivot >= NEAR_ALIAS): |D_gpu - D_oracle| <= TOL * chi2_0;
  * near-alias bins (oracle relative pivot < NEAR_ALIAS, i.e. nearly singular
    normal equations where Delta chi^2 is not a continuous function of the
    data): only the bounds 0 <= D <= chi2_0 (1 + TOL) are required;
  * argmax: same bin, or the oracle's values at the two bins differ by at most
    TOL * chi2_0 (several bins can be correct up to the tolerance).
"""
from __future__ import annotations

import numpy as np

TOL = 1e-4
NEAR_ALIAS = 1e-8


def compare(d_gpu, d_or, piv_or, chi0, tol=TOL, near_alias=NEAR_ALIAS):
    """d_gpu, d_or, piv_or: [nbins, H] arrays on the same bins."""
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    near = piv_or < near_alias
    err = np.abs(d_gpu - d_or)
    strict = err[~near]
    out = dict(
        max_err_rel=float(strict.max() / chi0) if strict.size else 0.0,
        n_strict=int((~near).sum()),
        n_near_alias=int(near.sum()),
        near_bounds_ok=bool(np.all(d_gpu[near] >= -tol * chi0) and
                            np.all(d_gpu[near] <= chi0 * (1 + tol))),
        finite=bool(np.all(np.isfinite(d_gpu))),
    )
    out["ok"] = out["finite"] and out["near_bounds_ok"] and out["max_err_rel"] <= tol
    return out


def argmax_ok(j_gpu, j_or, d_or_row, chi0, bins=None, tol=TOL):
    """d_or_row: oracle values over `bins` (or all bins when bins is None)."""
    if j_gpu == j_or:
        return True
    if bins is None:
        return d_or_row[j_or] - d_or_row[j_gpu] <= tol * chi0
    idx = {int(b): k for k, b in enumerate(bins)}
    if j_gpu not in idx:
        return False
    return d_or_row[idx[j_or]] - d_or_row[idx[j_gpu]] <= tol * chi0


def sample_bins(N, n_random, seed, windows=(), half=64):
    """Random bins plus +-half windows around the given centre bins."""
    rng = np.random.default_rng(seed)
    b = set(rng.choice(N, size=min(n_random, N), replace=False).tolist())
    for c in windows:
        c = int(c)
        for j in range(max(0, c - half), min(N, c + half + 1)):
            b.add(j)
    return np.array(sorted(b), dtype=np.int64)
