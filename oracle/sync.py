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
