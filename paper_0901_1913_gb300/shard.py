"""Sharding of the periodogram over ranks (one process per GPU).

Neither form has a collective on the data path:

* Independent curves (batched surveys): each rank takes a contiguous range of
  curves, balanced by a cost proxy, and runs ``execute_batched`` on it.
* One long curve: the trial range [0, N) is split into contiguous bands
  [j_a, j_b).  Each rank plans its band as its own trial grid
  (f_min' = f_min + j_a df, N' = j_b - j_a), so it runs its own transforms and
  solves; nothing is exchanged but the per-band records (a few KB, one
  all-gather).  The merge takes, per H', the best record over bands (value,
  then lowest j) and the top-K local maxima of Delta chi^2_H over bands.  A
  band tests its edge bins for the local-maximum rule against one side only,
  so each band reports K + 2 candidates together with its first and last
  Delta chi^2_H values, and the merge re-tests edge candidates against the
  neighbouring band's boundary value.

The rank-to-work assignment and the merge are plain host logic; ``allgather``
is any callable that returns the list of every rank's object (for example a
wrapper of ``torch.distributed.all_gather_object``).
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np


def band_partition(N: int, world: int) -> list[tuple[int, int]]:
    """Contiguous bands [j_a, j_b) covering [0, N), sizes differing by <= 1."""
    if N < 1 or world < 1:
        raise ValueError("N and world must be positive")
    world = min(world, N)
    q, r = divmod(N, world)
    out, a = [], 0
    for k in range(world):
        b = a + q + (1 if k < r else 0)
        out.append((a, b))
        a = b
    return out


def curve_partition(costs: Sequence[float], world: int) -> list[tuple[int, int]]:
    """Contiguous curve ranges [c_a, c_b) with near-equal summed cost (greedy
    on the cumulative cost); every rank gets a range, possibly empty."""
    costs = np.asarray(costs, dtype=np.float64)
    C = costs.size
    if world < 1:
        raise ValueError("world must be positive")
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        c = int(np.searchsorted(cum, target, side="left"))
        c = min(max(c, cuts[-1]), C)
        cuts.append(c)
    cuts.append(C)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def band_curve_args(f_min: float, df: float, band: tuple[int, int]) -> tuple[float, int]:
    """(f_min', N') of a band's own trial grid."""
    ja, jb = band
    return f_min + ja * df, jb - ja


def band_record(band: tuple[int, int], best: list[dict], peaks: list[dict],
                first_last: tuple[float, float]) -> dict:
    """What a rank contributes to the merge: its records with global bin
    indices and the Delta chi^2_H values of its first and last bins."""
    ja, jb = band

    def glob(r):
        r = dict(r)
        if r["j"] >= 0:
            r["j"] = int(r["j"]) + ja
        return r

    return {"band": (int(ja), int(jb)), "best": [glob(b) for b in best],
            "peaks": [glob(p) for p in peaks if p["j"] >= 0],
            "first": float(first_last[0]), "last": float(first_last[1])}


def _key(r):
    return (-r["dchi2"], r["j"])


def merge_records(recs: list[dict], K: int) -> tuple[list[dict], list[dict]]:
    """Merge band records (any order) into (best[H'], peaks[K])."""
    recs = sorted(recs, key=lambda r: r["band"][0])
    for a, b in zip(recs, recs[1:]):
        if a["band"][1] != b["band"][0]:
            raise ValueError("bands do not tile the trial range")
    H = len(recs[0]["best"])
    best = []
    for h in range(H):
        cands = [r["best"][h] for r in recs if r["best"][h]["j"] >= 0]
        best.append(min(cands, key=_key) if cands else dict(recs[0]["best"][h], j=-1))
    peaks = []
    for i, r in enumerate(recs):
        ja, jb = r["band"]
        left = recs[i - 1]["last"] if i > 0 else None
        right = recs[i + 1]["first"] if i + 1 < len(recs) else None
        for p in r["peaks"]:
            if p["j"] == ja and left is not None and not p["dchi2"] > left:
                continue
            if p["j"] == jb - 1 and right is not None and not p["dchi2"] >= right:
                continue
            peaks.append(p)
    peaks.sort(key=_key)
    return best, peaks[:K]


def run_band(make_plan: Callable, f_min: float, df: float, N: int, K: int, rank: int,
             world: int, allgather: Callable[[object], list]):
    """Run this rank's band and merge the records of all ranks.

    make_plan(f_min', N', top_k) -> a plan object with execute() returning
    (dchi2 [H, N'], best, peaks, chi2_0) as ``_fc2.Plan`` does.  Returns
    (band, dchi2 of the band, merged best, merged peaks, chi2_0)."""
    bands = band_partition(N, world)
    if rank >= len(bands):
        rec = None
        band, d, chi0 = (N, N), None, None
    else:
        band = bands[rank]
        fm, nb = band_curve_args(f_min, df, band)
        with make_plan(fm, nb, K + 2) as plan:
            d, best, peaks, chi0 = plan.execute()
        d = np.asarray(d) if not hasattr(d, "cpu") else d
        row = d[-1]
        first_last = (float(row[0]), float(row[-1]))
        rec = band_record(band, best, peaks, first_last)
    recs = [r for r in allgather(rec) if r is not None]
    best, peaks = merge_records(recs, K)
    return band, d, best, peaks, chi0


def curve_slice(offsets, arrays: Sequence, per_curve: Sequence, rng: tuple[int, int]):
    """The CSR sub-batch of curves [c_a, c_b): rebased offsets, the sample
    arrays' slices and the per-curve arrays' slices."""
    ca, cb = rng
    offsets = np.asarray(offsets, dtype=np.int64)
    a, b = int(offsets[ca]), int(offsets[cb])
    sub_off = offsets[ca:cb + 1] - a
    return sub_off, [arr[a:b] for arr in arrays], [np.asarray(v)[ca:cb] for v in per_curve]


def run_curves(execute_batched: Callable, offsets, t, x, sigma, H, f_min, df, N, rank: int,
               world: int, **kw):
    """This rank's share of a batch (contiguous curves balanced by
    n_c + H_c N_c): returns ((c_a, c_b), execute_batched's result)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    C = offsets.size - 1
    H, f_min, df, N = (np.broadcast_to(np.asarray(v), (C,)) for v in (H, f_min, df, N))
    cost = np.diff(offsets) + H.astype(np.float64) * N
    rng = curve_partition(cost, world)[rank]
    if rng[1] <= rng[0]:
        return rng, None
    sub_off, (ts, xs, ss), (hs, fs, ds, ns) = curve_slice(offsets, (t, x, sigma),
                                                         (H, f_min, df, N), rng)
    return rng, execute_batched(sub_off, ts, xs, ss, hs, fs, ds, ns, **kw)
