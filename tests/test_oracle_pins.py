"""Pins for the CPU oracle: each checks it against something other than itself.

* SSSP: a published worked example (CLRS Fig. 24.6, with a hand-worked BSP
  trace), SciPy's Dijkstra, and a heap Dijkstra written here.
* CC: SciPy's connected components and a union-find written here.
* PageRank / PPR: closed forms (directed cycle, undirected star, in-star with a
  dangling centre), two-scalar recurrences for exactly 20 supersteps, and the
  fixed point from a dense linear solve.
* LP (mode-label propagation): closed-form traces on a clique, an oscillating
  pair under the 15-superstep cap, a directed in-star, a directed path
  (Jacobi order), a majority that is not the minimum (multi-edges count), a
  self-loop, and an undirected star.
Each family is chosen so a dropped term, a wrong sign/index or a transposed
operand in the oracle fails at least one test.
"""
import heapq
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import oracle
from paper_2203_13005_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = oracle.INF


# ------------------------------------------------------------------ helpers

def _clrs():
    edges, dist, changed = [], None, None
    for ln in open(os.path.join(GOLDEN, "clrs_sssp.txt")):
        if not ln.strip() or ln.startswith("#"):
            continue
        tok = ln.split()
        if tok[0] == "edge":
            edges.append(tuple(int(x) for x in tok[1:]))
        elif tok[0] == "dist":
            dist = [int(x) for x in tok[1:]]
        elif tok[0] == "changed":
            changed = [int(x) for x in tok[1:]]
    e = np.array(edges, dtype=np.uint32)
    return e[:, 0], e[:, 1], e[:, 2], dist, changed


def _scipy_dijkstra(n, src, dst, w, source):
    # csr_matrix sums duplicates, so keep the minimum weight per (u, v) first
    key = src.astype(np.int64) * n + dst.astype(np.int64)
    order = np.lexsort((w, key))
    key_s, w_s = key[order], w[order]
    first = np.ones(len(key_s), dtype=bool)
    first[1:] = key_s[1:] != key_s[:-1]
    k, ww = key_s[first], w_s[first].astype(np.float64)
    m = sp.csr_matrix((ww, (k // n, k % n)), shape=(n, n))
    d = csg.dijkstra(m, directed=True, indices=source)
    out = np.full(n, INF, dtype=np.uint64)
    fin = np.isfinite(d)
    out[fin] = d[fin].astype(np.uint64)
    return out.astype(np.uint32)


def _heap_dijkstra(n, src, dst, w, source):
    adj = [[] for _ in range(n)]
    for u, v, c in zip(src.tolist(), dst.tolist(), w.tolist()):
        adj[u].append((v, c))
    dist = [INF] * n
    dist[source] = 0
    pq = [(0, source)]
    while pq:
        d, u = heapq.heappop(pq)
        if d > dist[u]:
            continue
        for v, c in adj[u]:
            if d + c < dist[v]:
                dist[v] = d + c
                heapq.heappush(pq, (d + c, v))
    return np.array(dist, dtype=np.uint32)


def _min_id_components(n, src, dst):
    g = sp.csr_matrix((np.ones(len(src)), (src.astype(np.int64), dst.astype(np.int64))), shape=(n, n))
    _, lab = csg.connected_components(g, directed=True, connection="weak")
    rep = np.full(lab.max() + 1 if n else 0, n, dtype=np.int64)
    np.minimum.at(rep, lab, np.arange(n))
    return rep[lab].astype(np.uint32)


def _union_find(n, src, dst):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for u, v in zip(src.tolist(), dst.tolist()):
        a, b = find(u), find(v)
        if a != b:
            if a < b:
                parent[b] = a
            else:
                parent[a] = b
    return np.array([find(v) for v in range(n)], dtype=np.uint32)


def _random_graph(rng, n, m, wmax=20):
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, wmax + 1, m, dtype=np.uint32)
    return src, dst, w


# --------------------------------------------------------------------- SSSP

def test_sssp_clrs_worked_example():
    src, dst, w, dist, changed = _clrs()
    d, steps, ch = oracle.sssp(5, src, dst, w, 0)
    assert d.tolist() == dist
    assert steps == len(changed) and ch.tolist() == changed


@pytest.mark.parametrize("seed", range(6))
def test_sssp_vs_dijkstra_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(0, 4 * n + 1))
    src, dst, w = _random_graph(rng, n, m)
    # include self-loops and duplicates on purpose
    if m:
        src[: m // 10] = dst[: m // 10]
    s = int(rng.integers(0, n))
    d, steps, _ = oracle.sssp(n, src, dst, w, s)
    assert np.array_equal(d, _heap_dijkstra(n, src, dst, w, s))
    assert np.array_equal(d, _scipy_dijkstra(n, src, dst, w, s))
    assert steps >= 1


def test_sssp_degenerate():
    # no edges: one superstep, nothing changes
    d, steps, ch = oracle.sssp(4, [], [], [], 2)
    assert d.tolist() == [INF, INF, 0, INF] and steps == 1 and ch.tolist() == [0]
    # source without out-edges, others unreachable
    d, steps, _ = oracle.sssp(3, [1], [2], [5], 0)
    assert d.tolist() == [0, INF, INF] and steps == 1
    # a path: one more vertex per superstep, then a no-change superstep
    n = 6
    src = np.arange(n - 1, dtype=np.uint32)
    d, steps, ch = oracle.sssp(n, src, src + 1, np.full(n - 1, 3, dtype=np.uint32), 0)
    assert d.tolist() == [0, 3, 6, 9, 12, 15] and steps == n and ch.tolist() == [1] * (n - 1) + [0]


def test_sssp_monotone_steps():
    rng = np.random.default_rng(7)
    n, m = 200, 900
    src, dst, w = _random_graph(rng, n, m)
    cur = np.full(n, INF, dtype=np.uint32)
    cur[0] = 0
    for _ in range(n + 1):
        nxt, c = oracle.sssp_step(n, src, dst, w, cur)
        assert np.all(nxt <= cur)
        assert c == int(np.sum(nxt != cur))
        cur = nxt
        if c == 0:
            break
    assert np.array_equal(cur, oracle.sssp(n, src, dst, w, 0)[0])


def test_sssp_rmat16_vs_dijkstra():
    wl = synth.SSSP_RMAT16
    src, dst, w = wl.edges()
    d, steps, _ = oracle.sssp(wl.n_vertices, src, dst, w, 0)
    assert np.array_equal(d, _scipy_dijkstra(wl.n_vertices, src, dst, w, 0))
    assert 5 < steps < 200


# ----------------------------------------------------------------------- CC

@pytest.mark.parametrize("seed", range(5))
def test_cc_vs_union_find_and_scipy(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 400))
    m = int(rng.integers(0, n + 1))
    a = rng.integers(0, n, m, dtype=np.uint32)
    b = rng.integers(0, n, m, dtype=np.uint32)
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    lab, steps, _ = oracle.cc(n, src, dst)
    assert np.array_equal(lab, _union_find(n, src, dst))
    assert np.array_equal(lab, _min_id_components(n, src, dst))


def test_cc_er_scaled_vs_scipy():
    n, m = 1 << 15, 1 << 17
    src, dst = synth.erdos_renyi(n, m // 2, 3)
    lab, steps, ch = oracle.cc(n, src, dst)
    assert np.array_equal(lab, _min_id_components(n, src, dst))
    assert ch[-1] == 0 and np.all(ch[:-1] > 0)


def test_cc_directed_reads_in_edges():
    # one direction only: label flows along edges, not against them
    lab, steps, _ = oracle.cc(3, [0, 1], [1, 2])   # 0 -> 1 -> 2
    assert lab.tolist() == [0, 0, 0] and steps == 3
    lab, steps, _ = oracle.cc(3, [2, 1], [1, 0])   # 2 -> 1 -> 0: smaller labels never move
    assert lab.tolist() == [0, 1, 2] and steps == 1


# ----------------------------------------------------------------- PageRank

D = 0.85


def test_pagerank_directed_cycle_uniform():
    for n in (1, 2, 5, 97):
        src = np.arange(n, dtype=np.uint32)
        dst = (src + 1) % n
        r, l1, dang = oracle.pagerank(n, src, dst, D, 20)
        assert np.allclose(r, 1.0 / n, rtol=1e-14, atol=0)
        assert np.all(dang == 0) and np.all(l1 < 1e-14)


def _star_recurrence(k, steps, dangling_centre):
    n = k + 1
    x = y = 1.0 / n
    for _ in range(steps):
        if dangling_centre:   # leaves -> centre only; centre's mass spread uniformly
            x, y = (1 - D) / n + D * (k * y + x / n), (1 - D) / n + D * (x / n)
        else:                 # undirected star: centre <-> each leaf
            x, y = (1 - D) / n + D * k * y, (1 - D) / n + D * x / k
    return x, y


@pytest.mark.parametrize("k", [1, 3, 7, 50])
def test_pagerank_undirected_star(k):
    n = k + 1
    leaves = np.arange(1, n, dtype=np.uint32)
    src = np.concatenate([np.zeros(k, np.uint32), leaves])
    dst = np.concatenate([leaves, np.zeros(k, np.uint32)])
    r, _, dang = oracle.pagerank(n, src, dst, D, 20)
    x, y = _star_recurrence(k, 20, False)
    assert abs(r[0] - x) < 1e-13 * x and np.allclose(r[1:], y, rtol=1e-13, atol=0)
    assert np.all(dang == 0)
    r_inf, _, _ = oracle.pagerank(n, src, dst, D, 400)
    assert abs(r_inf[0] - (1 + D * k) / (n * (1 + D))) < 1e-14
    assert abs(r_inf.sum() - 1) < 1e-13


@pytest.mark.parametrize("k", [1, 3, 7, 50])
def test_pagerank_in_star_dangling_centre(k):
    n = k + 1
    leaves = np.arange(1, n, dtype=np.uint32)
    src, dst = leaves, np.zeros(k, np.uint32)
    r, _, dang = oracle.pagerank(n, src, dst, D, 20)
    x, y = _star_recurrence(k, 20, True)
    assert abs(r[0] - x) < 1e-13 * x and np.allclose(r[1:], y, rtol=1e-13, atol=0)
    assert dang[0] == pytest.approx(1.0 / n, rel=1e-15)
    r_inf, _, _ = oracle.pagerank(n, src, dst, D, 400)
    assert abs(r_inf[0] - (1 + D * (n - 1)) / (n + D * (n - 1))) < 1e-14
    assert abs(r_inf[1] - (1 - D + D * r_inf[0]) / n) < 1e-14


def _google_fixed_point(n, src, dst):
    outdeg = np.bincount(src, minlength=n).astype(np.float64)
    M = np.zeros((n, n))
    for u, v in zip(src.tolist(), dst.tolist()):
        M[v, u] += 1.0 / outdeg[u]
    M[:, outdeg == 0] = 1.0 / n
    return np.linalg.solve(np.eye(n) - D * M, np.full(n, (1 - D) / n))


@pytest.mark.parametrize("seed", range(4))
def test_pagerank_fixed_point_linear_solve(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 120))
    m = int(rng.integers(1, 3 * n))
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    r, l1, _ = oracle.pagerank(n, src, dst, D, 400)
    assert np.allclose(r, _google_fixed_point(n, src, dst), rtol=1e-11, atol=1e-15)
    assert abs(r.sum() - 1) < 1e-12
    assert l1[-1] < 1e-20 + 1e-12 * l1[0]


def test_pagerank_step_matches_run():
    rng = np.random.default_rng(5)
    n, m = 300, 1500
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    r = np.full(n, 1.0 / n)
    dangs = []
    for _ in range(20):
        r, dng, _ = oracle.pagerank_step(n, src, dst, r, D)
        dangs.append(dng)
    r2, _, dang2 = oracle.pagerank(n, src, dst, D, 20)
    assert np.array_equal(r, r2) and np.allclose(dangs, dang2, rtol=0, atol=0)


def test_pagerank_rmat_mass_conserved():
    src, dst = synth.rmat(12, 1 << 16, 9)
    r, l1, dang = oracle.pagerank(4096, src, dst, D, 20)
    assert abs(r.sum() - 1) < 1e-12
    assert np.all(dang > 0) and l1[-1] < l1[0]


# ---------------------------------------------------------------------- PPR

def test_ppr_cycle_closed_form():
    n, t = 7, 20
    src = np.arange(n, dtype=np.uint32)
    dst = (src + 1) % n
    r = oracle.ppr(n, src, dst, 0, D, t)
    want = np.zeros(n)
    for k in range(t):
        want[k % n] += (1 - D) * D**k
    want[t % n] += D**t
    assert np.allclose(r, want, rtol=1e-14, atol=1e-17)


@pytest.mark.parametrize("seed", range(3))
def test_ppr_fixed_point_linear_solve(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 100))
    m = int(rng.integers(1, 3 * n))
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    s = int(rng.integers(0, n))
    outdeg = np.bincount(src, minlength=n).astype(np.float64)
    M = np.zeros((n, n))
    for u, v in zip(src.tolist(), dst.tolist()):
        M[v, u] += 1.0 / outdeg[u]
    M[s, outdeg == 0] = 1.0
    e = np.zeros(n)
    e[s] = 1 - D
    want = np.linalg.solve(np.eye(n) - D * M, e)
    r = oracle.ppr(n, src, dst, s, D, 400)
    assert np.allclose(r, want, rtol=1e-11, atol=1e-15)
    assert abs(r.sum() - 1) < 1e-12


# ------------------------------------------------------------------------ LP

def _undirected(pairs):
    a = np.array([p[0] for p in pairs], np.uint32)
    b = np.array([p[1] for p in pairs], np.uint32)
    return np.concatenate([a, b]), np.concatenate([b, a])


@pytest.mark.parametrize("k", [4, 7])
def test_lp_clique_trace(k):
    # K_k on ids 10..10+k-1 inside 30 vertices. Superstep 1: every neighbour
    # label occurs once, so the minimum wins: vertex 10 takes 11, the others
    # take 10. Superstep 2: vertex 10 sees k-1 tens, the others see one 11 and
    # k-2 >= 2 tens: all take 10. Superstep 3 changes nothing.
    n, base = 30, 10
    src, dst = _undirected([(base + i, base + j) for i in range(k) for j in range(i + 1, k)])
    l1, c1 = oracle.lp_step(n, src, dst, np.arange(n, dtype=np.uint32))
    exp1 = np.arange(n, dtype=np.uint32)
    exp1[base] = base + 1
    exp1[base + 1:base + k] = base
    assert np.array_equal(l1, exp1) and c1 == k
    labels, steps, changed = oracle.lp(n, src, dst)
    exp = np.arange(n, dtype=np.uint32)
    exp[base:base + k] = base
    assert np.array_equal(labels, exp)
    assert steps == 3 and list(changed) == [k, 1, 0]


def test_lp_pair_oscillates_to_the_cap():
    # two vertices joined both ways swap labels every superstep: never quiet
    src, dst = _undirected([(0, 1)])
    for cap in (1, 2, 15):
        labels, steps, changed = oracle.lp(3, src, dst, max_steps=cap)
        assert steps == cap and list(changed) == [2] * cap
        assert list(labels) == ([1, 0, 2] if cap % 2 else [0, 1, 2])


def test_lp_in_star_reads_in_edges():
    # leaves 1..5 -> centre 0: the centre sees five distinct labels and takes
    # the smallest (1); the leaves have no in-edges and keep theirs
    src = np.arange(1, 6, dtype=np.uint32)
    dst = np.zeros(5, np.uint32)
    labels, steps, changed = oracle.lp(6, src, dst)
    assert list(labels) == [1, 1, 2, 3, 4, 5]
    assert steps == 2 and list(changed) == [1, 0]


def test_lp_path_is_jacobi():
    # 0 -> 1 -> 2 -> 3: superstep t moves label 0 one hop (an in-place update
    # would carry it to the end in one superstep)
    src = np.array([0, 1, 2], np.uint32)
    dst = np.array([1, 2, 3], np.uint32)
    l1, _ = oracle.lp_step(4, src, dst, np.arange(4, dtype=np.uint32))
    assert list(l1) == [0, 0, 1, 2]
    labels, steps, changed = oracle.lp(4, src, dst)
    assert list(labels) == [0, 0, 0, 0]
    assert steps == 4 and list(changed) == [3, 2, 1, 0]


def test_lp_majority_beats_minimum():
    # vertex 9 receives 5 twice (a multi-edge) and 3 once: the mode is 5
    src = np.array([5, 5, 3], np.uint32)
    dst = np.array([9, 9, 9], np.uint32)
    l1, c1 = oracle.lp_step(10, src, dst, np.arange(10, dtype=np.uint32))
    assert l1[9] == 5 and c1 == 1
    # with one edge from 5, 5 and 3 tie and the smaller label wins
    l1, _ = oracle.lp_step(10, src[1:], dst[1:], np.arange(10, dtype=np.uint32))
    assert l1[9] == 3


def test_lp_self_loop_counts():
    # 7 -> 7 twice and 2 -> 7: the own label arrives twice and wins; with one
    # self-loop the tie goes to the smaller label 2
    l1, _ = oracle.lp_step(8, np.array([7, 7, 2], np.uint32), np.array([7, 7, 7], np.uint32),
                           np.arange(8, dtype=np.uint32))
    assert l1[7] == 7
    l1, _ = oracle.lp_step(8, np.array([7, 2], np.uint32), np.array([7, 7], np.uint32),
                           np.arange(8, dtype=np.uint32))
    assert l1[7] == 2


@pytest.mark.parametrize("k", [3, 6])
def test_lp_undirected_star_trace(k):
    # centre 0, leaves 1..k: the leaves take 0 and the centre the smallest
    # leaf label 1; then the leaves take 1 and the centre sees k zeros
    # (takes 0); the two labels swap between centre and leaves from then on
    src, dst = _undirected([(0, i) for i in range(1, k + 1)])
    n = k + 1
    labels, steps, changed = oracle.lp(n, src, dst, max_steps=15)
    assert steps == 15
    assert list(changed) == [k + 1] + [k + 1] * 14
    # after an odd number of supersteps: centre 1, leaves 0
    assert labels[0] == 1 and np.all(labels[1:] == 0)
    labels, _, _ = oracle.lp(n, src, dst, max_steps=4)
    assert labels[0] == 0 and np.all(labels[1:] == 1)


def test_lp_result_labels_come_from_in_neighbours():
    # invariant on a random graph: every new label is the old one (no
    # in-edges) or the label of an in-neighbour, and no other label reaches
    # the vertex more often
    rng = np.random.default_rng(4)
    n = 300
    src = rng.integers(0, n, 900, dtype=np.uint32)
    dst = rng.integers(0, n, 900, dtype=np.uint32)
    l0 = rng.integers(0, 20, n, dtype=np.uint32)
    l1, _ = oracle.lp_step(n, src, dst, l0)
    for v in range(n):
        msgs = l0[src[dst == v]]
        if len(msgs) == 0:
            assert l1[v] == l0[v]
            continue
        vals, cnt = np.unique(msgs, return_counts=True)
        assert l1[v] in vals
        assert cnt[vals == l1[v]][0] == cnt.max()
        assert l1[v] == vals[cnt == cnt.max()].min()
