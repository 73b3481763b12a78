"""Push-direction and direction-switching supersteps of SSSP and CC against
the oracle: the same values and the same changed counts after every
superstep (Jacobi order), whichever direction each superstep takes, on one
partition and on several (where a push relaxes each partition's in-edges
from its own changed vertices and from its cached copies of changed remote
vertices, and the exchange's upload lists stay the oracle's); frontier work
items cut at 32 out-edges; values set between supersteps."""
import numpy as np
import pytest

import oracle
from oracle import sync as osync
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu

DIRS = {"pull": gxp.GXP_DIR_PULL, "push": gxp.GXP_DIR_PUSH, "auto": gxp.GXP_DIR_AUTO}


def _rmat(scale, ef=16, seed=0x51, w_hi=100):
    src, dst = synth.rmat(scale, ef << scale, seed)
    w = synth.weights(len(src), 1, w_hi, seed)
    return 1 << scale, src, dst, w


@pytest.mark.parametrize("parts,keep_ids", [(1, False), (1, True), (2, False), (8, False)])
@pytest.mark.parametrize("direction", ["pull", "push", "auto"])
def test_sssp_every_superstep_matches_oracle(direction, parts, keep_ids):
    n, src, dst, w = _rmat(12)
    with gxp.Context(0, direction=DIRS[direction], keep_ids=keep_ids) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 0)
        d = np.full(n, gxp.INF, np.uint32)
        d[0] = 0
        steps = 0
        while True:
            d_ref, ch_ref = oracle.sssp_step(n, src, dst, w, d)
            ch = c.superstep()
            steps += 1
            assert ch == ch_ref, f"superstep {steps}"
            assert np.array_equal(c.values(), d_ref), f"superstep {steps}"
            d = d_ref
            if ch_ref == 0:
                break
        st = c.stats()
        assert st["supersteps"] == steps
        if direction == "pull":
            assert st["push_supersteps"] == 0
        elif direction == "push":
            assert st["push_supersteps"] == steps
        else:
            assert 0 < st["push_supersteps"] < steps   # the first and last supersteps push, the bulk pulls


@pytest.mark.parametrize("push_div", [1, 4, 8, 64])
@pytest.mark.parametrize("direction", ["push", "auto"])
def test_sssp_run_matches_oracle(direction, push_div):
    wl = synth.SSSP_RMAT16
    src, dst, w = wl.edges()
    n = wl.n_vertices
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 0)
    with gxp.Context(0, direction=DIRS[direction], push_div=push_div) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst, w)
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == steps_ref
        assert np.array_equal(c.values(), d_ref)
        st = c.stats()
        assert st["supersteps"] == steps_ref
        # pushed supersteps scan only their frontier's out-edges
        if st["push_supersteps"]:
            assert st["edges_scanned"] < st["supersteps"] * len(src)
        # a second run from another source reuses the out-edge copy
        s2 = int(np.flatnonzero(np.bincount(src, minlength=n))[7])
        d2, st2, _ = oracle.sssp(n, src, dst, w, s2)
        assert c.run(gxp.GXP_ALGO_SSSP, s2) == st2
        assert np.array_equal(c.values(), d2)


@pytest.mark.parametrize("parts", [1, 2, 8])
@pytest.mark.parametrize("direction", ["pull", "push", "auto"])
def test_cc_every_superstep_matches_oracle(direction, parts):
    rng = np.random.default_rng(9)
    n = 3000
    a = rng.integers(0, n, 2500, dtype=np.uint32)
    b = rng.integers(0, n, 2500, dtype=np.uint32)
    src, dst = np.concatenate([a, b]), np.concatenate([b, a])
    bounds = [n * p // parts for p in range(parts + 1)]
    _, _, trace = osync.min_label_sync_trace(n, src, dst, bounds, "cc")
    with gxp.Context(0, direction=DIRS[direction]) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_CC)
        lab = np.arange(n, dtype=np.uint32)
        steps = 0
        while True:
            l_ref, ch_ref = oracle.cc_step(n, src, dst, lab)
            ch = c.superstep()
            steps += 1
            assert ch == ch_ref, f"superstep {steps}"
            assert np.array_equal(c.values(), l_ref), f"superstep {steps}"
            if parts > 1:   # the exchange uploads the oracle's pairs whichever direction ran
                uploads, skipped = trace[steps - 1]
                for p in range(parts):
                    ids, vals, sk = c.sync(p)
                    assert sk == skipped and np.array_equal(ids, uploads[p][0]), (steps, p)
                    assert np.array_equal(vals, uploads[p][1]), (steps, p)
            lab = l_ref
            if ch_ref == 0:
                break
        if direction == "push":
            assert c.stats()["push_supersteps"] == steps
        elif direction == "auto":
            # with partitions the first supersteps (up to 1529 of 3000 labels
            # changing) pull without listing their changed vertices; the
            # listing resumes once the frontier shrinks, and the tail pushes
            assert 0 < c.stats()["push_supersteps"] < steps
        labels, steps_ref, _ = oracle.cc(n, src, dst)
        assert steps == steps_ref
        assert c.run(gxp.GXP_ALGO_CC) == steps_ref
        assert np.array_equal(c.values(), labels)


@pytest.mark.parametrize("direction", ["push", "auto"])
def test_item_boundaries(direction):
    # sources with 1, 31, 32, 33, 64, 65 and 1000 out-edges (work items of 32),
    # vertices without out-edges, and vertices the source does not reach
    rng = np.random.default_rng(3)
    n = 5000
    s, d = [], []
    hubs = {1: 1, 2: 31, 3: 32, 4: 33, 5: 64, 6: 65, 7: 1000}
    for v, k in hubs.items():
        s += [v] * k
        d += list(rng.integers(100, 4000, k))
    s += [0] * 7
    d += list(hubs)
    s += [9, 10]
    d += [10, 11]            # 9 -> 10 -> 11 unreachable from 0
    s += list(rng.integers(100, 4000, 3000))
    d += list(rng.integers(100, 4999, 3000))
    src, dst = np.array(s, np.uint32), np.array(d, np.uint32)
    w = rng.integers(1, 200, len(src), dtype=np.uint32)
    d_ref, steps_ref, ch_ref = oracle.sssp(n, src, dst, w, 0)
    with gxp.Context(0, direction=DIRS[direction]) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 0)
        for t in range(steps_ref):
            assert c.superstep() == ch_ref[t]
        assert np.array_equal(c.values(), d_ref)
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == steps_ref


@pytest.mark.parametrize("parts", [1, 3])
@pytest.mark.parametrize("direction", ["pull", "push", "auto"])
def test_values_set_between_supersteps(direction, parts):
    n, src, dst, w = _rmat(11, seed=0x77)
    with gxp.Context(0, direction=DIRS[direction]) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst, w)
        c.begin(gxp.GXP_ALGO_SSSP, 5)
        c.superstep()
        c.superstep()
        d = c.values()
        # raise some distances and lower others, then continue to convergence
        rng = np.random.default_rng(1)
        d = d.copy()
        idx = rng.choice(n, 200, replace=False)
        d[idx[:100]] = np.minimum(d[idx[:100]], rng.integers(0, 50, 100).astype(np.uint32))
        d[idx[100:]] = gxp.INF
        c.set_values(d)
        cur = d
        while True:
            ref, ch_ref = oracle.sssp_step(n, src, dst, w, cur)
            assert c.superstep() == ch_ref
            assert np.array_equal(c.values(), ref)
            cur = ref
            if ch_ref == 0:
                break


def test_degenerate_graphs_push():
    e = np.zeros(0, np.uint32)
    for n in (1, 4):
        with gxp.Context(0, direction=gxp.GXP_DIR_PUSH) as c:
            c.create_graph(n, 1)
            c.load_coo(e, e, e)
            assert c.run(gxp.GXP_ALGO_SSSP, n - 1) == 1
            d = c.values()
            assert d[n - 1] == 0 and np.all(np.delete(d, n - 1) == gxp.INF)
            assert c.run(gxp.GXP_ALGO_CC) == 1
            assert np.array_equal(c.values(), np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("cache_slots", [0, 16, gxp.GXP_CACHE_NONE])
@pytest.mark.parametrize("direction", ["push", "auto"])
def test_partitioned_runs_and_caches(direction, cache_slots):
    """Whole runs over 4 partitions from two sources, with the LRU cache on or
    off; PageRank and label propagation on the same context pull as before."""
    n, src, dst, w = _rmat(10, seed=0x33)
    d_ref, steps_ref, _ = oracle.sssp(n, src, dst, w, 0)
    s2 = int(np.flatnonzero(np.bincount(src, minlength=n))[11])
    d2, st2, _ = oracle.sssp(n, src, dst, w, s2)
    with gxp.Context(0, direction=DIRS[direction], cache_slots=cache_slots) as c:
        c.create_graph(n, 4)
        c.load_coo(src, dst, w)
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == steps_ref
        assert np.array_equal(c.values(), d_ref)
        if direction == "push":
            assert c.stats()["push_supersteps"] == steps_ref
        else:
            assert c.stats()["push_supersteps"] > 0
        assert c.run(gxp.GXP_ALGO_SSSP, s2) == st2
        assert np.array_equal(c.values(), d2)
        c.run(gxp.GXP_ALGO_PAGERANK, max_steps=2)     # other algorithms are unaffected
        r_ref, _, _ = oracle.pagerank(n, src, dst, 0.85, 2)
        assert np.max(np.abs(c.values() - r_ref) / r_ref) <= 1e-4


def test_invalid_direction():
    with pytest.raises(gxp.GxpError) as ei:
        gxp.Context(0, direction=7)
    assert ei.value.code == gxp.GXP_E_INVAL


@pytest.mark.parametrize("direction", ["pull", "push", "auto"])
def test_long_runs_and_step_limits(direction):
    # a weighted path plus chords: more supersteps than one device-driven
    # launch holds (32), and runs cut short by max_steps
    rng = np.random.default_rng(11)
    n = 150
    a = np.arange(n - 1, dtype=np.uint32)
    src = np.concatenate([a, rng.integers(0, n, 40, dtype=np.uint32)])
    dst = np.concatenate([a + 1, rng.integers(0, n, 40, dtype=np.uint32)])
    w = np.concatenate([np.ones(n - 1, np.uint32), rng.integers(200, 400, 40, dtype=np.uint32)])
    d_ref, steps_ref, ch_ref = oracle.sssp(n, src, dst, w, 0)
    assert steps_ref > 64
    with gxp.Context(0, direction=DIRS[direction]) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst, w)
        assert c.run(gxp.GXP_ALGO_SSSP, 0) == steps_ref
        assert np.array_equal(c.values(), d_ref)
        st = c.stats()
        assert st["supersteps"] == steps_ref and st["last_changed"] == 0
        for cap in (1, 5, 32, 33, 70):
            d_cap, s_cap, _ = oracle.sssp(n, src, dst, w, 0, max_steps=cap)
            assert c.run(gxp.GXP_ALGO_SSSP, 0, max_steps=cap) == s_cap == cap
            assert np.array_equal(c.values(), d_cap)
            assert c.stats()["last_changed"] == ch_ref[cap - 1]
        # CC over both directions of the path
        s2, d2 = np.concatenate([src, dst]), np.concatenate([dst, src])
        labels, cc_steps, _ = oracle.cc(n, s2, d2)
    with gxp.Context(0, direction=DIRS[direction]) as c:
        c.create_graph(n, 1)
        c.load_coo(s2, d2)
        assert c.run(gxp.GXP_ALGO_CC) == cc_steps
        assert np.array_equal(c.values(), labels)
        # manual supersteps after a run continue from its state
        c.begin(gxp.GXP_ALGO_CC)
        for _ in range(3):
            c.superstep()
        l3, _, _ = oracle.cc(n, s2, d2, max_steps=3)
        assert np.array_equal(c.values(), l3)
