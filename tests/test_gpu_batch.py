"""GPU parity of the batched multi-source SSSP (gxp_sssp_batch) against the
CPU oracle, source by source, bit for bit — resident and streamed edges,
pipelined or not, replayed from a CUDA graph or not, fixed or autotuned
block sizes."""
import numpy as np
import pytest

import oracle
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu


def _graph(scale, seed=0x67700004):
    wl = synth.MSSSP_RMAT24.scaled(scale)
    src, dst, w = wl.edges()
    return wl.n_vertices, src, dst, w, seed


def _check(n, src, dst, w, sources, dist):
    for k, s in enumerate(sources):
        ref, _, _ = oracle.sssp(n, src, dst, w, int(s))
        assert np.array_equal(dist[:, k], ref), f"source {s} (slot {k})"


@pytest.fixture(scope="module")
def g12():
    n, src, dst, w, seed = _graph(12)
    sources = synth.sources_with_out_edges(n, src, 64, seed)
    return n, src, dst, w, sources


def _ctx(n, src, dst, w):
    c = gxp.Context(0)
    c.create_graph(n, 1)
    c.load_coo(src, dst, w)
    return c


def test_batch_resident_64_sources(g12):
    n, src, dst, w, sources = g12
    with _ctx(n, src, dst, w) as c:
        dist, rep = c.sssp_batch(sources)
        assert rep["supersteps"] >= 2
        assert rep["persistent"] == 1   # resident edges: one persistent cooperative launch
    _check(n, src, dst, w, sources, dist)


@pytest.mark.parametrize("streamed", [False, True])
def test_batch_counts_active_edges(g12, streamed):
    # the report's active in-edges (those whose source is in the frontier):
    # the first superstep's frontier is the sources, so one superstep walks
    # exactly their out-edges; a whole run walks at least that and at most
    # every edge per superstep
    n, src, dst, w, sources = g12
    outdeg = np.bincount(src, minlength=n)
    first = int(outdeg[np.unique(sources)].sum())
    with _ctx(n, src, dst, w) as c:
        _, rep1 = c.sssp_batch(sources, streamed=streamed, block_edges=3000 if streamed else 0, max_steps=1)
        _, rep = c.sssp_batch(sources, streamed=streamed, block_edges=3000 if streamed else 0)
    assert rep1["supersteps"] == 1 and rep1["active_edges"] == first
    assert first <= rep["active_edges"] <= rep["supersteps"] * len(src)


@pytest.mark.parametrize("pipelined,use_graph", [(True, False), (False, False), (True, True)])
def test_batch_streamed_small_blocks(g12, pipelined, use_graph):
    n, src, dst, w, sources = g12
    with _ctx(n, src, dst, w) as c:
        ref, _ = c.sssp_batch(sources)
        dist, rep = c.sssp_batch(sources, streamed=True, pipelined=pipelined, block_edges=3000,
                                 use_graph=use_graph)
        assert rep["blocks"] >= 10
        assert np.array_equal(dist, ref)
        dist2, _ = c.sssp_batch(sources, streamed=True, pipelined=pipelined, block_edges=3000,
                                use_graph=use_graph)
        assert np.array_equal(dist2, ref)
    _check(n, src, dst, w, sources[:8], dist)


def test_batch_autotuned_block_size():
    n, src, dst, w, seed = _graph(15)
    sources = synth.sources_with_out_edges(n, src, 64, seed)
    with _ctx(n, src, dst, w) as c:
        ref, _ = c.sssp_batch(sources)
        dist, rep = c.sssp_batch(sources, streamed=True, block_edges=0, use_graph=True)
        assert np.array_equal(dist, ref)
        assert rep["k1"] > 0 and rep["k2"] > 0 and rep["a"] > 0
        assert rep["blocks"] >= 1 and rep["model_block_edges"] > 0 and rep["sweep_best_ms"] > 0
    _check(n, src, dst, w, sources[:4], dist)


def test_batch_split_rows_and_few_sources():
    # an in-star whose centre has far more in-edges than one work unit, plus a path
    k = 3000
    leaves = np.arange(1, k + 1, dtype=np.uint32)
    src = np.concatenate([leaves, leaves[:-1]])
    dst = np.concatenate([np.zeros(k, np.uint32), leaves[1:]])
    w = (np.arange(len(src), dtype=np.uint32) % 17) + 1
    n = k + 1
    sources = np.array([1, 5, 2999], dtype=np.uint32)
    with _ctx(n, src, dst, w) as c:
        dist, _ = c.sssp_batch(sources)
        dist_s, _ = c.sssp_batch(sources, streamed=True, block_edges=700)
    assert dist.shape == (n, 3) and np.array_equal(dist, dist_s)
    _check(n, src, dst, w, sources, dist)


def test_batch_errors(g12):
    n, src, dst, w, sources = g12
    with _ctx(n, src, dst, w) as c:
        with pytest.raises(gxp.GxpError) as ei:
            c.sssp_batch(np.arange(65, dtype=np.uint32))
        assert ei.value.code == gxp.GXP_E_INVAL
        with pytest.raises(gxp.GxpError) as ei:
            c.sssp_batch(np.array([n], dtype=np.uint32))
        assert ei.value.code == gxp.GXP_E_INVAL
    with gxp.Context(0) as c:
        c.create_graph(n, 2)
        c.load_coo(src, dst, w)
        with pytest.raises(gxp.GxpError) as ei:
            c.sssp_batch(sources[:2])
        assert ei.value.code == gxp.GXP_E_UNSUPPORTED


@pytest.mark.slow
def test_batch_rmat24_streamed_vs_oracle_and_single_source_runs():
    """The full batched workload (R-MAT 24, 64 sources, edges streamed through
    the pipeline shuffle): 4 sources against the oracle, and all 64 columns
    against single-source runs of the superstep engine on the same GPU."""
    wl = synth.MSSSP_RMAT24
    src, dst, w = wl.edges()
    n = wl.n_vertices
    sources = synth.sources_with_out_edges(n, src, 64, wl.seed)
    with _ctx(n, src, dst, w) as c:
        dist, rep = c.sssp_batch(sources, streamed=True, use_graph=True)
    _check(n, src, dst, w, sources[:4], dist)
    with gxp.Context(0) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst, w)
        for j, s in enumerate(sources):
            c.run(gxp.GXP_ALGO_SSSP, source=int(s))
            assert np.array_equal(c.values(), dist[:, j]), j


def test_batch_wide_weights_unpacked_edges():
    # weights above 255 do not fit the 4-byte packed edge: the 8-byte layout runs
    rng = np.random.default_rng(77)
    n, m = 3000, 40000
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, 100000, m, dtype=np.uint32)
    sources = synth.sources_with_out_edges(n, src, 16, 5)
    with _ctx(n, src, dst, w) as c:
        dist, _ = c.sssp_batch(sources)
        dist_s, _ = c.sssp_batch(sources, streamed=True, block_edges=5000)
    assert np.array_equal(dist, dist_s)
    _check(n, src, dst, w, sources, dist)


def test_batch_tune_cache_skips_the_measurements(tmp_path, g12):
    """With a tune cache, the first autotuned run measures and stores its
    coefficients and block size; the next run on the same shape and GPU reads
    them (tune_from_cache) and gives the same distances."""
    n, src, dst, w, sources = g12
    path = str(tmp_path / "tune.json")
    with _ctx(n, src, dst, w) as c:
        d1, r1 = c.sssp_batch(sources, streamed=True, tune_cache=path)
        d2, r2 = c.sssp_batch(sources, streamed=True, tune_cache=path)
    assert r1["tune_from_cache"] == 0 and r2["tune_from_cache"] == 1
    assert r2["block_edges"] == r1["block_edges"] and r2["k2"] == r1["k2"] and r2["a"] == r1["a"]
    assert np.array_equal(d1, d2)
    _check(n, src, dst, w, sources[:3], d2)
    import json
    data = json.load(open(path))
    assert len(data) == 1 and next(iter(data)).startswith(f"sssp_batch V={n} ")
