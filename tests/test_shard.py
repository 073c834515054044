"""Host logic of the multi-rank sharding (no GPU): partitions, the record
merge, and a two-rank gloo run whose bands are evaluated by the oracle and
whose merged records must equal the unsharded ones exactly."""
import os
import socket

import numpy as np
import pytest

from paper_0901_1913_gb300 import shard, synth


def band_records_like_library(d, K):
    """Stand-in for the library's records on one band: argmax per row (lowest
    j on ties) and top-K local maxima of the last row (> left, >= right, edges
    one-sided), by value then j."""
    H, N = d.shape
    best = []
    for h in range(H):
        j = int(np.argmax(d[h]))
        best.append({"j": j, "dchi2": float(d[h, j]), "H": h + 1})
    r = d[-1]
    cand = []
    for j in range(N):
        left = j == 0 or r[j] > r[j - 1]
        right = j == N - 1 or r[j] >= r[j + 1]
        if left and right:
            cand.append({"j": j, "dchi2": float(r[j]), "H": H})
    cand.sort(key=lambda p: (-p["dchi2"], p["j"]))
    return best, cand[:K]


def test_band_partition_tiles():
    for N in (1, 7, 64, 1000):
        for world in (1, 2, 3, 8):
            b = shard.band_partition(N, world)
            assert b[0][0] == 0 and b[-1][1] == N
            assert all(x[1] == y[0] for x, y in zip(b, b[1:]))
            sizes = [y - x for x, y in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1


def test_curve_partition_balances():
    rng = np.random.default_rng(0)
    costs = rng.lognormal(7.0, 1.0, 500)
    for world in (1, 2, 4, 8):
        parts = shard.curve_partition(costs, world)
        assert parts[0][0] == 0 and parts[-1][1] == costs.size
        assert all(x[1] == y[0] for x, y in zip(parts, parts[1:]))
        loads = [costs[a:b].sum() for a, b in parts]
        assert max(loads) <= costs.sum() / world + costs.max()


def test_merge_rejects_edge_peaks_that_are_not_global_maxima():
    # bands [0,4) and [4,8); row values make bin 4 a band-local edge peak but not
    # a global one (its left neighbour, bin 3, is larger)
    row = np.array([0.0, 1.0, 2.0, 5.0, 4.0, 3.0, 6.0, 1.0])
    recs = []
    for a, b in shard.band_partition(8, 2):
        d = row[a:b][None, :]
        best, peaks = band_records_like_library(d, 3 + 2)
        recs.append(shard.band_record((a, b), best, peaks, (d[-1, 0], d[-1, -1])))
    best, peaks = shard.merge_records(recs, 3)
    gbest, gpeaks = band_records_like_library(row[None, :], 3)
    assert [p["j"] for p in peaks] == [p["j"] for p in gpeaks] == [6, 3]
    assert best[0]["j"] == gbest[0]["j"] == 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        c = synth.short_curve(n=160, N=96)
        K = 4

        class OraclePlan:
            """Evaluates a band with the oracle (exact per bin)."""

            def __init__(self, f_min, N, top_k):
                self.f_min, self.N, self.top_k = f_min, N, top_k

            def __enter__(self):
                return self

            def __exit__(self, *a):
                pass

            def execute(self):
                d = np.asarray(oracle.periodogram(c.t, c.x, c.sigma, c.H, self.f_min, c.df,
                                                  self.N, threads=1)).T
                best, peaks = band_records_like_library(d, self.top_k)
                return d, best, peaks, 1.0

        def allgather(obj):
            out = [None] * world
            dist.all_gather_object(out, obj)
            return out

        band, d, best, peaks, _ = shard.run_band(OraclePlan, c.f_min, c.df, c.N, K, rank, world,
                                                 allgather)
        if rank == 0:
            full = OraclePlan(c.f_min, c.N, K).execute()
            q.put(([b["j"] for b in best], [p["j"] for p in peaks],
                   [b["j"] for b in full[1]], [p["j"] for p in full[2]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_band_merge_equals_unsharded():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    best_j, peak_j, full_best_j, full_peak_j = got
    assert best_j == full_best_j
    assert peak_j == full_peak_j


def test_curve_shards_cover_the_batch_once():
    b = synth.survey_batch(seed=3, C=40, N=1 << 10, n_median=300.0, n_hi=1000)
    seen = []

    def fake_execute(off, t, x, s, H, fm, df, N, **kw):
        # the sub-batch is a consistent CSR slice of the full batch
        assert off[0] == 0 and off[-1] == t.size == x.size == s.size
        assert len(H) == len(fm) == len(df) == len(N) == off.size - 1
        return float(t.sum())

    total = 0.0
    for world in (1, 3):
        total = 0.0
        for rank in range(world):
            rng, r = shard.run_curves(fake_execute, b.offsets, b.t, b.x, b.sigma, b.H, b.f_min,
                                      b.df, b.N, rank, world)
            seen.append(rng)
            total += r if r is not None else 0.0
        assert abs(total - b.t.sum()) <= 1e-9 * abs(b.t.sum())
