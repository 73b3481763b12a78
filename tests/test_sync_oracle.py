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


# ---------------------------------------------------------------- LRU cache

def _golden_lru():
    path = __file__.replace("test_sync_oracle.py", "golden/lru_trace_6v.txt")
    kv = {}
    for ln in open(path):
        ln = ln.strip()
        if not ln or ln.startswith("#"):
            continue
        k, v = ln.split(":", 1)
        kv[k.strip()] = v.strip()
    edges = [tuple(int(x) for x in e.split()) for e in kv["edges"].split(",")]
    after = []
    t = 1
    while f"after {t}" in kv:
        row = []
        for part in kv[f"after {t}"].split(";"):
            ids, d = part.strip().split("|")
            row.append(([int(x) for x in ids.split()[1:]], int(d)))
        after.append(row)
        t += 1
    return (np.array([e[0] for e in edges], np.uint32), np.array([e[1] for e in edges], np.uint32),
            [int(x) for x in kv["bounds"].split()], int(kv["capacity"]),
            [int(x) for x in kv["before"].split()], after)


def test_lru_hand_trace():
    src, dst, bounds, cap, before, after = _golden_lru()
    lab, steps, trace0, trace = sync.lru_trace(6, src, dst, bounds, cap)
    assert lab.tolist() == [0] * 6 and steps == 4
    assert trace0 == before
    assert [[(k, d) for k, d in row] for row in trace] == after


def test_lru_weight_rule():
    # decay by half, rise by reads when used, saturate at W_MAX; evict lowest, ties evict higher id
    kept, w, d = sync.lru_boundary({7, 9}, {7: 10, 9: 3}, [9, 11], {7: 1, 9: 4, 11: 5}, 2)
    # 7: 10//2 = 5; 9: 3//2 + 4 = 5; 11 enters with 5 -> all tie at 5: keep 7, 9 (lower ids)
    assert kept == {7, 9} and w == {7: 5, 9: 5} and d == 1
    kept, w, d = sync.lru_boundary(set(), {}, [1, 2], {1: 70000, 2: 3}, 1)
    assert kept == {1} and w == {1: sync.W_MAX} and d == 2
    kept, w, d = sync.lru_boundary({1}, {1: sync.W_MAX}, [1], {1: 70000}, 1)
    assert w == {1: sync.W_MAX} and d == 0
    # capacity 0: every use downloads, nothing is kept
    kept, w, d = sync.lru_boundary(set(), {}, [4, 5], {4: 1, 5: 1}, 0)
    assert kept == set() and d == 2


def test_lru_unbounded_downloads_each_copy_once_and_invariants():
    wl = synth.CC_ER24_P8.scaled(10)
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    bounds = [n * p // 4 for p in range(5)]
    ghosts = sync.reads_per_copy(n, src, dst, bounds)
    big = max(len(g) for g, _ in ghosts)
    lab, steps, trace0, trace = sync.lru_trace(n, src, dst, bounds, big)
    ref, rsteps, _ = oracle.cc(n, src, dst)
    assert np.array_equal(lab, ref) and steps == rsteps
    # room for every copy: each is downloaded once, at its first use (superstep 1, CC)
    assert trace0 == [len(g) for g, _ in ghosts]
    assert all(d == 0 for row in trace for _, d in row)
    for cap in (1, 7, 50):
        _, _, t0, tr = sync.lru_trace(n, src, dst, bounds, cap)
        for p, (g, _) in enumerate(ghosts):
            assert t0[p] == len(g)
            for row in tr:
                kept, d = row[p]
                assert len(kept) <= cap and set(kept) <= set(g.tolist())
