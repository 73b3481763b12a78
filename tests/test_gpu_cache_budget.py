"""Synchronization caching under a budget (cache_slots): every partition
keeps its most-read remote copies cached and downloads the others again
after every superstep. Values, changed counts, upload lists and skip flags
are the same at every budget; the downloads follow from the ghost counts."""
import numpy as np
import pytest

import oracle
from oracle import sync as osync
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu


def _ghost_counts(n, src, dst, parts):
    """Distinct remote sources read by each partition (its cached copies when unbudgeted)."""
    b = np.array([n * p // parts for p in range(parts + 1)])
    owner_d = np.searchsorted(b, dst, side="right") - 1
    owner_s = np.searchsorted(b, src, side="right") - 1
    return [len(np.unique(src[(owner_d == p) & (owner_s != p)])) for p in range(parts)]


@pytest.mark.parametrize("budget", [0, 40, 1, gxp.GXP_CACHE_NONE])
@pytest.mark.parametrize("algo", ["sssp", "cc"])
def test_budget_changes_nothing_but_downloads(algo, budget):
    rng = np.random.default_rng(17)
    n, m, parts = 3000, 12000, 4
    src = rng.integers(0, n, m, dtype=np.uint32)
    dst = rng.integers(0, n, m, dtype=np.uint32)
    w = rng.integers(1, 60, m, dtype=np.uint32)
    if algo == "cc":
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        w = None
    b = [n * p // parts for p in range(parts + 1)]
    ref, steps, trace = osync.min_label_sync_trace(n, src, dst, b, algo, w=w, source=0)
    ghosts = _ghost_counts(n, src, dst, parts)
    if budget == 0:
        kept = ghosts
    elif budget == gxp.GXP_CACHE_NONE:
        kept = [0] * parts
    else:
        kept = [min(g, budget) for g in ghosts]
    with gxp.Context(0, cache_slots=budget) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP if algo == "sssp" else gxp.GXP_ALGO_CC, 0)
        for t in range(steps):
            c.superstep()
            uploads, skipped = trace[t]
            for p in range(parts):
                ids, vals, sk = c.sync(p)
                assert sk == skipped, (t, p)
                assert np.array_equal(ids, uploads[p][0]) and np.array_equal(vals, uploads[p][1]), (t, p)
        assert np.array_equal(c.values(), ref)
        st = c.stats()
        assert st["cache_downloads"] == steps * (sum(ghosts) - sum(kept))


def test_budget_with_lp_and_runs():
    wl = synth.CC_ER24_P8.scaled(14)
    src, dst, _ = wl.edges()
    n = wl.n_vertices
    labels, steps, _ = oracle.lp(n, src, dst)
    cc_ref, cc_steps, _ = oracle.cc(n, src, dst)
    for budget in (0, 500, gxp.GXP_CACHE_NONE):
        with gxp.Context(0, cache_slots=budget) as c:
            c.create_graph(n, wl.parts)
            c.load_coo(src, dst)
            assert c.run(gxp.GXP_ALGO_LP, max_steps=oracle.LP_MAX_STEPS) == steps
            assert np.array_equal(c.values(), labels)
            assert c.run(gxp.GXP_ALGO_CC) == cc_steps
            assert np.array_equal(c.values(), cc_ref)
            if budget == 0:
                assert c.stats()["cache_downloads"] == 0
            else:
                assert c.stats()["cache_downloads"] > 0
