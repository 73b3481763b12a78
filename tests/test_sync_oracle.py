"""Pins for the synchronization caching/skipping oracle (Section III-B)."""
import numpy as np

import oracle
from oracle import sync
from paper_2203_13005_gb300 import synth


def test_path_two_partitions_hand_trace():
    # undirected path 0-1-2-3, partitions {0,1} | {2,3}
    src = np.array([0, 1, 1, 2, 2, 3], dtype=np.uint32)
    dst = np.array([1, 0, 2, 1, 3, 2], dtype=np.uint32)
    bset = sync.boundary_sets(4, src, dst, [0, 2, 4])
    assert [b.tolist() for b in bset] == [[1], [2]]
    lab, steps, trace = sync.min_label_sync_trace(4, src, dst, [0, 2, 4])
    assert lab.tolist() == [0, 0, 0, 0] and steps == 4
    # worked by hand: labels [0,0,1,2] -> [0,0,0,1] -> [0,0,0,0] -> same
    want = [
        ([([1], [0]), ([2], [1])], False),
        ([([], []), ([2], [0])], False),
        ([([], []), ([], [])], True),
        ([([], []), ([], [])], True),
    ]
    for (ups, skipped), (wups, wskip) in zip(trace, want):
        assert skipped == wskip
        for (ids, vals), (wi, wv) in zip(ups, wups):
            assert ids.tolist() == wi and vals.tolist() == wv


def test_disconnected_partitions_always_skip():
    # two cliques, one per partition, no edge between them
    a = [(u, v) for u in range(4) for v in range(4) if u != v]
    b = [(u + 4, v + 4) for u, v in a]
    e = np.array(a + b, dtype=np.uint32)
    lab, steps, trace = sync.min_label_sync_trace(8, e[:, 0], e[:, 1], [0, 4, 8])
    assert lab.tolist() == [0] * 4 + [4] * 4
    assert all(skipped for _, skipped in trace)


def _boundary_by_loops(n, src, dst, bounds):
    own = lambda v: max(p for p in range(len(bounds) - 1) if bounds[p] <= v)
    out = [set() for _ in range(len(bounds) - 1)]
    for u, v in zip(src.tolist(), dst.tolist()):
        if own(u) != own(v):
            out[own(u)].add(u)
    return [sorted(s) for s in out]


def test_boundary_sets_vs_loops():
    rng = np.random.default_rng(3)
    n, m = 60, 200
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    bounds = [0, 13, 13, 40, 60]          # includes an empty partition
    got = sync.boundary_sets(n, src, dst, bounds)
    assert [g.tolist() for g in got] == _boundary_by_loops(n, src, dst, bounds)


def test_partitioned_trace_equals_unpartitioned_run():
    n = 1 << 12
    src, dst = synth.erdos_renyi(n, 1 << 13, 17)
    bounds = [i * n // 8 for i in range(9)]
    lab, steps, trace = sync.min_label_sync_trace(n, src, dst, bounds)
    lab2, steps2, ch = oracle.cc(n, src, dst)
    assert np.array_equal(lab, lab2) and steps == steps2
    # an upload is a subset of that superstep's changed vertices
    for t, (ups, _) in enumerate(trace):
        assert sum(len(i) for i, _ in ups) <= ch[t]


def test_sssp_trace():
    wl = synth.SSSP_RMAT16.scaled(10)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    bounds = [0, 300, 700, n]
    d, steps, trace = sync.min_label_sync_trace(n, src, dst, bounds, algo="sssp", w=w, source=0)
    d2, steps2, _ = oracle.sssp(n, src, dst, w, 0)
    assert np.array_equal(d, d2) and steps == steps2
    assert trace[-1][1]  # nothing changes in the last superstep, so nothing to sync
