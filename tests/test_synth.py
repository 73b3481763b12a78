"""Seeded input generators: published SplitMix64 vectors, determinism, shapes."""
import os

import numpy as np
import pytest

from paper_2203_13005_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for seed, i, val in rows:
        assert synth.u64(int(seed), int(i)) == int(val)


def test_stream_matches_scalar():
    s = synth.stream_u64(99, 5, 7)
    assert [int(x) for x in s] == [synth.u64(99, 5 + i) for i in range(7)]
    u = synth.stream_unit(99, 5, 7)
    assert np.all((u >= 0) & (u < 1))
    assert np.array_equal(u, (s >> np.uint64(11)).astype(np.float64) * 2.0**-53)


def test_rmat_deterministic_and_shaped():
    s1, d1 = synth.rmat(12, 1 << 16, 7)
    s2, d2 = synth.rmat(12, 1 << 16, 7)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    assert s1.max() < 4096 and d1.max() < 4096
    # top bit of (src, dst) follows the quadrant probabilities (a, b, c, d)
    top_s = (s1 >> 11) & 1
    top_d = (d1 >> 11) & 1
    n = len(s1)
    frac = {q: np.mean((top_s == q[0]) & (top_d == q[1])) for q in [(0, 0), (0, 1), (1, 0), (1, 1)]}
    assert abs(frac[(0, 0)] - 0.57) < 0.01
    assert abs(frac[(0, 1)] - 0.19) < 0.01
    assert abs(frac[(1, 0)] - 0.19) < 0.01
    assert abs(frac[(1, 1)] - 0.05) < 0.01
    s3, _ = synth.rmat(12, 1 << 16, 8)
    assert not np.array_equal(s1, s3)


def test_rmat_prefix_stable():
    # edge i depends only on (seed, i): a shorter run is a prefix of a longer one
    s1, d1 = synth.rmat(10, 1000, 3)
    s2, d2 = synth.rmat(10, 5000, 3)
    assert np.array_equal(s1, s2[:1000]) and np.array_equal(d1, d2[:1000])


def test_er_symmetric_no_self_loops():
    s, d = synth.erdos_renyi(1000, 20000, 11)
    assert len(s) == 40000
    assert np.all(s != d)
    assert np.array_equal(s[0::2], d[1::2]) and np.array_equal(d[0::2], s[1::2])
    assert s.max() < 1000
    # uniform endpoints: each vertex appears ~40 times
    c = np.bincount(s, minlength=1000)
    assert 20 < c.mean() < 60


def test_er_tiny_n():
    s, d = synth.erdos_renyi(2, 100, 5)
    assert np.all(s != d) and set(np.unique(s)) <= {0, 1}


def test_weights_range():
    w = synth.weights(100000, 1, 100, 3)
    assert w.min() == 1 and w.max() == 100
    assert abs(w.mean() - 50.5) < 0.5


def test_sample_sources():
    s, d = synth.rmat(10, 1 << 14, 1)
    src = synth.sources_with_out_edges(1024, s, 64, 4)
    assert len(set(src.tolist())) == 64
    outdeg = np.bincount(s, minlength=1024)
    assert np.all(outdeg[src] > 0)
    assert np.array_equal(src, synth.sources_with_out_edges(1024, s, 64, 4))
    with pytest.raises(ValueError):
        synth.sample_vertices(10, np.zeros(10, dtype=bool), 1, 0)


def test_poisson_arrivals():
    t = synth.poisson_arrivals(2000.0, 2.0, 5)
    assert np.all(np.diff(t) > 0) and t[-1] < 2.0
    assert abs(len(t) - 4000) < 4 * np.sqrt(4000)


def test_workload_sizes():
    w = synth.SSSP_RMAT16
    assert (w.n_vertices, w.n_edges, w.w_lo, w.w_hi) == (65536, 1048576, 1, 100)
    assert synth.PAGERANK_RMAT22.n_vertices == 4194304 and synth.PAGERANK_RMAT22.n_edges == 67108864
    assert synth.CC_ER24_P8.n_edges == 268435456 and synth.CC_ER24_P8.parts == 8
    assert synth.MSSSP_RMAT24.n_vertices == 16777216 and synth.MSSSP_RMAT24.w_hi == 255
    small = w.scaled(8)
    assert small.n_vertices == 256 and small.n_edges == 4096
    s22 = synth.SSSP_RMAT22
    assert (s22.n_vertices, s22.n_edges, s22.w_lo, s22.w_hi, s22.seed) == (4194304, 67108864, 1, 100, 0x67700006)
    cl = synth.SSSP_CLUSTERED24_P8
    assert (cl.kind, cl.n_vertices, cl.n_edges, cl.parts, cl.p_cross, cl.w_hi) == (
        "clustered", 16777216, 268435456, 8, 1e-5, 100)
    cls = cl.scaled(12)   # the recipe at another size keeps its kind, blocks and crossing rate
    assert (cls.kind, cls.n_vertices, cls.n_edges, cls.parts, cls.p_cross) == ("clustered", 4096, 65536, 8, 1e-5)
    src, dst, wts = cls.edges()
    assert len(src) == len(wts) == 65536 and wts.min() >= 1 and wts.max() <= 100
    # every workload has its own seed
    seeds = [x.seed for x in (synth.SSSP_RMAT16, synth.PAGERANK_RMAT22, synth.CC_ER24_P8, synth.MSSSP_RMAT24,
                              synth.SSSP_RMAT22, synth.SSSP_CLUSTERED24_P8)] + [g.seed for g in synth.SERVE_GRAPHS]
    assert len(set(seeds)) == len(seeds)


def test_clustered_blocks_and_crossing_fraction():
    n, k, m, pc = 4000, 8, 50000, 0.01
    src, dst = synth.clustered(n, k, m, pc, 0x1234)
    assert len(src) == 2 * m
    # pairs are stored in both directions, without self-loops
    assert np.array_equal(src[0::2], dst[1::2]) and np.array_equal(dst[0::2], src[1::2])
    assert np.all(src != dst) and src.max() < n
    block = lambda x: (x.astype(np.int64) * k) // n   # the default partition cut
    cross = (block(src) != block(dst)).mean()
    assert abs(cross - pc) < 0.003
    # every block is used, about evenly
    counts = np.bincount(block(src[0::2]), minlength=k)
    assert counts.min() > 0.8 * m / k
    # counter-based: the same seed gives the same graph, another seed another
    s2, d2 = synth.clustered(n, k, m, pc, 0x1234)
    assert np.array_equal(src, s2) and np.array_equal(dst, d2)
    s3, _ = synth.clustered(n, k, m, pc, 0x1235)
    assert not np.array_equal(src, s3)
    # no crossing at all when p_cross = 0
    s0, d0 = synth.clustered(n, k, 5000, 0.0, 7)
    assert np.all(block(s0) == block(d0))
