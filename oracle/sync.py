"""Synchronization caching and skipping between partitions (Section III-B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Vertices are owned by contiguous id ranges: partition p owns
[bounds[p], bounds[p+1]). Each partition computes on its own vertices and
reads cached copies of the remote source vertices of its in-edges.

* Lazy uploading (Algorithm 3): the global query queue is the union of what
  each partition needs from the others, i.e. every vertex with an out-edge
  into another partition ("boundary" vertices). After a superstep, partition
  p uploads to the global data queue only its vertices that both changed in
  that superstep and are in the query queue: changed(p) ∩ boundary(p),
  reported as (id, new value) pairs in ascending id order.
* Skipping (Section III-B3): when no updated vertex has an out-edge leaving
  its partition — every partition's upload is empty — the global exchange of
  that superstep is skipped.

Neither changes any vertex value: a partitioned Jacobi run with these rules
equals the unpartitioned one, superstep for superstep.
"""
from __future__ import annotations

import numpy as np

from . import cc_step, sssp_step


def owners(n: int, bounds) -> np.ndarray:
    bounds = np.asarray(bounds, dtype=np.int64)
    return (np.searchsorted(bounds, np.arange(n), side="right") - 1).astype(np.int64)


def boundary_sets(n: int, src, dst, bounds) -> list[np.ndarray]:
    """boundary(p): sorted ids owned by p with at least one out-edge to another partition."""
    own = owners(n, bounds)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    leaving = own[src] != own[dst]
    b = np.unique(src[leaving])
    return [b[(own[b] == p)] for p in range(len(bounds) - 1)]


def lazy_upload(prev: np.ndarray, cur: np.ndarray, boundary_p: np.ndarray):
    """(ids, values) uploaded by one partition after a superstep."""
    ids = boundary_p[cur[boundary_p] != prev[boundary_p]]
    return ids.astype(np.uint32), cur[ids]


def min_label_sync_trace(n, src, dst, bounds, algo="cc", w=None, source=0, max_steps=1 << 20):
    """Run the Jacobi min-propagation oracle (CC or SSSP) and record, per superstep,
    each partition's upload and whether the exchange is skipped.

    Returns (final values, steps, trace) with trace[t] = (uploads, skipped),
    uploads[p] = (ids, values).
    """
    bset = boundary_sets(n, src, dst, bounds)
    if algo == "cc":
        cur = np.arange(n, dtype=np.uint32)
    elif algo == "sssp":
        cur = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
        cur[source] = 0
    else:
        raise ValueError(algo)
    trace = []
    steps = 0
    for _ in range(max_steps):
        if algo == "cc":
            nxt, changed = cc_step(n, src, dst, cur)
        else:
            nxt, changed = sssp_step(n, src, dst, w, cur)
        steps += 1
        uploads = [lazy_upload(cur, nxt, bset[p]) for p in range(len(bounds) - 1)]
        skipped = all(len(ids) == 0 for ids, _ in uploads)
        trace.append((uploads, skipped))
        cur = nxt
        if changed == 0:
            break
    return cur, steps, trace


# ---------------------------------------------------------------- LRU cache
#
# LRU-based caching (Section III-B2), with the readings this oracle takes
# where the passage is silent or contradicts itself:
#  * A copy of remote vertex u is *used* by partition p in superstep t when
#    u is in that superstep's frontier: u changed in superstep t - 1 (superstep
#    1: every vertex for CC / LP / PageRank, the source for SSSP). Only then
#    does its value matter to p's computation.
#  * Weights are integers. Before superstep t, every copy that is cached or
#    used gets  W <- min(W_MAX, floor(W / 2) + reads_p(u) * [u used in t]),
#    where reads_p(u) counts p's in-edges from u: the weight decays by half
#    per superstep and rises with use. A copy entering the cache starts at 0
#    before that update.
#  * Every used copy that is not cached is downloaded (counted) and enters the
#    cache; when more than C copies are then held, the ones with the lowest
#    weights are evicted (the passage says "highest" in one sentence and
#    "lowest" in the next; the LRU sense is the lowest), ties going to the
#    higher vertex id. An evicted copy forgets its weight.
# None of this changes a value: a used copy is always fresh (downloaded, or
# refreshed by the lazy upload of the superstep that changed it).

W_MAX = 65535


def reads_per_copy(n, src, dst, bounds):
    """Per partition p: (ghost ids ascending, reads_p of each ghost)."""
    own = owners(n, bounds)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    out = []
    for p in range(len(bounds) - 1):
        sel = (own[dst] == p) & (own[src] != p)
        g, cnt = np.unique(src[sel], return_counts=True)
        out.append((g.astype(np.int64), cnt.astype(np.int64)))
    return out


def lru_boundary(kept: dict, weight: dict, used_ids, reads: dict, cap: int):
    """One boundary of one partition. kept: set of cached ids; weight: id ->
    weight of cached ids; used_ids: ids used by the coming superstep (subset of
    the partition's ghosts); reads: id -> reads_p. Returns (new kept set, new
    weights, downloads)."""
    used = set(int(u) for u in used_ids)
    downloads = len(used - kept)
    cand = kept | used
    w = {}
    for u in cand:
        old = weight.get(u, 0) if u in kept else 0
        w[u] = min(W_MAX, old // 2 + (reads[u] if u in used else 0))
    order = sorted(cand, key=lambda u: (-w[u], u))
    new_kept = set(order[:cap])
    return new_kept, {u: w[u] for u in new_kept}, downloads


def lru_trace(n, src, dst, bounds, cap, algo="cc", w=None, source=0, max_steps=1 << 20):
    """Jacobi min-label run (CC or SSSP) with each partition's LRU cache of
    capacity `cap`. Returns (values, steps, trace) with trace[t] = per
    partition (kept ids ascending after the boundary that follows superstep
    t + 1, downloads at that boundary), and the downloads of the boundary
    before superstep 1 as trace0."""
    ghosts = reads_per_copy(n, src, dst, bounds)
    P = len(bounds) - 1
    reads = [dict(zip(g.tolist(), c.tolist())) for g, c in ghosts]
    gsets = [set(g.tolist()) for g, _ in ghosts]
    if algo == "cc":
        cur = np.arange(n, dtype=np.uint32)
        frontier = set(range(n))
    else:
        cur = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
        cur[source] = 0
        frontier = {source}
    kept = [set() for _ in range(P)]
    wts = [dict() for _ in range(P)]
    trace0 = []
    for p in range(P):
        kept[p], wts[p], d = lru_boundary(kept[p], wts[p], sorted(gsets[p] & frontier), reads[p], cap)
        trace0.append(d)
    trace = []
    steps = 0
    for _ in range(max_steps):
        if algo == "cc":
            nxt, changed = cc_step(n, src, dst, cur)
        else:
            nxt, changed = sssp_step(n, src, dst, w, cur)
        steps += 1
        frontier = set(np.nonzero(nxt != cur)[0].tolist())
        row = []
        for p in range(P):
            kept[p], wts[p], d = lru_boundary(kept[p], wts[p], sorted(gsets[p] & frontier), reads[p], cap)
            row.append((sorted(kept[p]), d))
        trace.append(row)
        cur = nxt
        if changed == 0:
            break
    return cur, steps, trace0, trace
