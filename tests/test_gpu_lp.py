"""Label propagation (mode merge, Jacobi, 15-superstep cap) through the C-ABI
against the oracle: labels and changed counts after every superstep, on one
partition (renumbered or not) and on several, with rows in every in-degree
class (1..32, 33..256, 257..2048, hub rows cut into chunks of 2048 with a hash table),
ties, multi-edges, self-loops and graphs that never settle."""
import numpy as np
import pytest

import oracle
from paper_2203_13005_gb300 import gxp, synth

pytestmark = pytest.mark.gpu

CAP = oracle.LP_MAX_STEPS


def _mixed_graph(seed, n=12000):
    """Symmetric R-MAT core plus rows of 32, 33, 256, 257, 2048, 2049, 4097 and 9000 in-edges
    (sources drawn from a few hundred vertices: repeated labels early) and
    multi-edges / self-loops."""
    rng = np.random.default_rng(seed)
    s, d = synth.rmat(13, 8 << 13, seed)
    s, d = np.concatenate([s, d]), np.concatenate([d, s])
    extra_s, extra_d = [], []
    for v, k in ((9000, 32), (9001, 33), (9002, 2048), (9003, 2049), (9004, 9000), (9005, 4097), (9006, 256),
                 (9007, 257)):
        extra_s.append(rng.integers(0, 400, k, dtype=np.uint32))
        extra_d.append(np.full(k, v, np.uint32))
    extra_s.append(np.array([9100, 9100, 9101], np.uint32))   # self-loops, multi-edge
    extra_d.append(np.array([9100, 9100, 9100], np.uint32))
    src = np.concatenate([s] + extra_s).astype(np.uint32)
    dst = np.concatenate([d] + extra_d).astype(np.uint32)
    return n, src, dst


@pytest.mark.parametrize("keep_ids", [False, True])
@pytest.mark.parametrize("parts", [1, 4])
def test_every_superstep_matches_oracle(parts, keep_ids):
    if parts > 1 and keep_ids:
        pytest.skip("partitions keep input ids anyway")
    n, src, dst = _mixed_graph(21)
    with gxp.Context(0, keep_ids=keep_ids) as c:
        c.create_graph(n, parts)
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_LP)
        lab = np.arange(n, dtype=np.uint32)
        for t in range(CAP):
            ref, ch_ref = oracle.lp_step(n, src, dst, lab)
            ch = c.superstep()
            assert ch == ch_ref, f"superstep {t + 1}"
            assert np.array_equal(c.values(), ref), f"superstep {t + 1}"
            lab = ref
            if ch_ref == 0:
                break
        labels, steps, changed = oracle.lp(n, src, dst)
        assert c.run(gxp.GXP_ALGO_LP, max_steps=CAP) == steps
        assert np.array_equal(c.values(), labels)
        assert c.stats()["last_changed"] == changed[-1]


def test_rmat_run_and_partition_counts_agree():
    wl = synth.SSSP_RMAT16
    s, d, _ = wl.edges()
    src, dst = np.concatenate([s, d]), np.concatenate([d, s])
    n = wl.n_vertices
    labels, steps, changed = oracle.lp(n, src, dst)
    for parts in (1, 8):
        with gxp.Context(0) as c:
            c.create_graph(n, parts)
            c.load_coo(src, dst)
            assert c.run(gxp.GXP_ALGO_LP, max_steps=CAP) == steps
            assert np.array_equal(c.values(), labels)
            st = c.stats()
            assert st["supersteps"] == steps and st["last_changed"] == changed[-1]
            if parts > 1:
                assert st["syncs_done"] + st["syncs_skipped"] == steps


def test_oscillating_pair_runs_to_the_cap():
    src = np.array([0, 1], np.uint32)
    dst = np.array([1, 0], np.uint32)
    with gxp.Context(0) as c:
        c.create_graph(3, 1)
        c.load_coo(src, dst)
        assert c.run(gxp.GXP_ALGO_LP, max_steps=CAP) == CAP
        assert list(c.values()) == [1, 0, 2]
        assert c.stats()["last_changed"] == 2


def test_degenerate_graphs():
    e = np.zeros(0, np.uint32)
    for n in (1, 5):
        with gxp.Context(0) as c:
            c.create_graph(n, 1)
            c.load_coo(e, e)
            assert c.run(gxp.GXP_ALGO_LP, max_steps=CAP) == 1
            assert np.array_equal(c.values(), np.arange(n, dtype=np.uint32))


def test_values_set_between_supersteps():
    n, src, dst = _mixed_graph(5, n=10000)
    with gxp.Context(0) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_LP)
        c.superstep()
        rng = np.random.default_rng(2)
        lab = rng.integers(0, 50, n).astype(np.uint32)   # few labels: long runs, hub tables hit hard
        c.set_values(lab)
        for _ in range(6):
            ref, ch_ref = oracle.lp_step(n, src, dst, lab)
            assert c.superstep() == ch_ref
            assert np.array_equal(c.values(), ref)
            lab = ref


def test_template_checked():
    src = np.array([0], np.uint32)
    dst = np.array([1], np.uint32)
    with gxp.Context(0) as c:
        c.create_graph(2, 1)
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_LP)
        with pytest.raises(gxp.GxpError) as ei:
            c.superstep(template=(gxp.GXP_GEN_LABEL, gxp.GXP_MERGE_MIN, gxp.GXP_APPLY_MIN))
        assert ei.value.code == gxp.GXP_E_UNSUPPORTED
        c.superstep()
        assert list(c.values()) == [0, 0]


@pytest.mark.slow
def test_wide_labels():
    # more than 2^27 vertices: the (row, label) keys no longer fit 32 bits;
    # cliques, a star and a hub among the ids above 2^27
    n = (1 << 27) + 64
    base = 1 << 27
    rng = np.random.default_rng(8)
    s, d = [], []
    for c0 in (base, base + 20):
        for i in range(8):
            for j in range(8):
                if i != j:
                    s.append(c0 + i)
                    d.append(c0 + j)
    for leaf in range(base + 40, base + 50):
        s += [leaf, base + 39]
        d += [base + 39, leaf]
    hub_src = rng.integers(base, n, 5000)
    s += list(hub_src)
    d += [base + 63] * len(hub_src)
    src, dst = np.array(s, np.uint32), np.array(d, np.uint32)
    with gxp.Context(0) as c:
        c.create_graph(n, 1)
        c.load_coo(src, dst)
        c.begin(gxp.GXP_ALGO_LP)
        lab = np.arange(n, dtype=np.uint32)
        for t in range(4):
            ref, ch_ref = oracle.lp_step(n, src, dst, lab)
            assert c.superstep() == ch_ref, f"superstep {t + 1}"
            got = c.values()
            assert np.array_equal(got[base:], ref[base:]) and np.array_equal(got[:base], ref[:base])
            lab = ref
