"""The CPU baselines bench.py times (oracle/cpu_baselines.c) compute what the
oracle computes: all-cores pull PageRank, all-cores pull min-label supersteps,
binary-heap Dijkstra and union-find, on small seeded graphs. They are not the
oracle and no GPU parity check uses them; this only keeps the timed baselines
honest."""
import numpy as np

import oracle
from oracle import cpu_baselines as cb
from paper_2203_13005_gb300 import synth


def test_pagerank_pull_matches_oracle():
    wl = synth.PAGERANK_RMAT22.scaled(12)
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    cp, s, _ = cb.csc(n, src, dst)
    cb.set_threads(4)
    r = cb.pagerank_pull(n, cp, s, np.bincount(src, minlength=n), 0.85, 20)
    ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 20)
    assert np.max(np.abs(r - ref) / ref) < 1e-12


def test_minlabel_pull_sssp_and_cc_match_oracle():
    wl = synth.SSSP_RMAT16.scaled(11)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    cp, s, cw = cb.csc(n, src, dst, w)
    d0 = np.full(n, 0xFFFFFFFF, np.uint32)
    d0[0] = 0
    d, steps = cb.minlabel_pull(n, cp, s, cw, d0)
    ref, rsteps, _ = oracle.sssp(n, src, dst, w, 0)
    assert np.array_equal(d, ref) and steps == rsteps
    es, ed = synth.erdos_renyi(1 << 12, 1 << 12, 3)
    cp, s, _ = cb.csc(1 << 12, es, ed)
    lab, steps = cb.minlabel_pull(1 << 12, cp, s, None, np.arange(1 << 12, dtype=np.uint32))
    ref, rsteps, _ = oracle.cc(1 << 12, es, ed)
    assert np.array_equal(lab, ref) and steps == rsteps


def test_dijkstra_and_union_find_match_oracle():
    wl = synth.SSSP_RMAT16.scaled(11)
    src, dst, w = wl.edges()
    n = wl.n_vertices
    rp, cd, cw = cb.csr(n, src, dst, w)
    ref, _, _ = oracle.sssp(n, src, dst, w, 0)
    assert np.array_equal(cb.dijkstra(n, rp, cd, cw, 0), ref)
    es, ed = synth.erdos_renyi(1 << 12, 1 << 11, 9)
    ref, _, _ = oracle.cc(1 << 12, es, ed)
    assert np.array_equal(cb.union_find(1 << 12, es, ed), ref)


def test_host_cores_and_threads():
    assert cb.host_cores() >= 1
    assert cb.set_threads(2) == 2
