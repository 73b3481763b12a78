"""Seeded synthetic graph inputs (R-MAT, Erdős–Rényi, weights, sources).

Pure input generation, no step of the superstep method: the CUDA path, the
CPU oracle, the tests and ``bench.py`` all draw their inputs here. The random
stream is SplitMix64 used as a counter-based generator (see ``csrc/synth.c``
for the exact definition), so every array is a pure function of its seed.

The named workloads below mirror the paper's evaluation inputs (Section V-A,
Table I: power-law social graphs such as Orkut, LiveJournal and Twitter, plus
uniform "synthetic" data for the skipping experiment of Section V-B) with
seeded stand-ins: R-MAT (a,b,c,d) = (.57,.19,.19,.05), edge factor 16, for the
power-law graphs and Erdős–Rényi G(n, m) for the uniform ones.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_synth()
        lib = C.CDLL(path)
        u64, u32, dbl, p = C.c_uint64, C.c_uint32, C.c_double, C.c_void_p
        lib.gxs_u64.restype = u64
        lib.gxs_u64.argtypes = [u64, u64]
        lib.gxs_fill_u64.argtypes = [u64, u64, u64, p]
        lib.gxs_fill_unit.argtypes = [u64, u64, u64, p]
        lib.gxs_rmat.argtypes = [u32, u64, dbl, dbl, dbl, u64, p, p]
        lib.gxs_er.argtypes = [u64, u64, u64, p, p]
        lib.gxs_clustered.argtypes = [u64, u32, u64, dbl, u64, p, p]
        lib.gxs_weights.argtypes = [u64, u32, u32, u64, p]
        lib.gxs_sample.restype = u32
        lib.gxs_sample.argtypes = [u64, p, u32, u64, p, p]
        lib.gxs_omp_threads.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# Stream separation: each kind of draw uses the base seed xor a fixed tag.
WEIGHT_TAG = 0x7765696768747321  # "weights!"
SOURCE_TAG = 0x736F757263657321  # "sources!"
ARRIVE_TAG = 0x6172726976616C21  # "arrival!"


def u64(seed: int, i: int) -> int:
    return int(_load().gxs_u64(seed & (2**64 - 1), i))


def stream_u64(seed: int, i0: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().gxs_fill_u64(seed & (2**64 - 1), i0, n, _ptr(out))
    return out


def stream_unit(seed: int, i0: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().gxs_fill_unit(seed & (2**64 - 1), i0, n, _ptr(out))
    return out


def rmat(scale: int, n_edges: int, seed: int, a=0.57, b=0.19, c=0.19):
    """R-MAT COO edges (src, dst) as uint32 arrays over 2**scale vertices."""
    src = np.empty(n_edges, dtype=np.uint32)
    dst = np.empty(n_edges, dtype=np.uint32)
    _load().gxs_rmat(scale, n_edges, a, b, c, seed & (2**64 - 1), _ptr(src), _ptr(dst))
    return src, dst


def erdos_renyi(n: int, m_pairs: int, seed: int):
    """G(n, m) pairs stored in both directions: 2*m_pairs directed edges."""
    if n < 2:
        raise ValueError("Erdős–Rényi needs n >= 2")
    src = np.empty(2 * m_pairs, dtype=np.uint32)
    dst = np.empty(2 * m_pairs, dtype=np.uint32)
    _load().gxs_er(n, m_pairs, seed & (2**64 - 1), _ptr(src), _ptr(dst))
    return src, dst


def clustered(n: int, blocks: int, m_pairs: int, p_cross: float, seed: int):
    """Planted-partition pairs in `blocks` contiguous id blocks (the default
    partition cut), a fraction p_cross of them joining two different blocks,
    stored in both directions: 2*m_pairs directed edges."""
    if blocks < 1 or n < 2 * blocks:
        raise ValueError("clustered graph needs n >= 2 * blocks")
    src = np.empty(2 * m_pairs, dtype=np.uint32)
    dst = np.empty(2 * m_pairs, dtype=np.uint32)
    _load().gxs_clustered(n, blocks, m_pairs, float(p_cross), seed & (2**64 - 1), _ptr(src), _ptr(dst))
    return src, dst


def weights(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    w = np.empty(n, dtype=np.uint32)
    _load().gxs_weights(n, lo, hi, (seed ^ WEIGHT_TAG) & (2**64 - 1), _ptr(w))
    return w


def sample_vertices(n: int, eligible: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k distinct vertices, uniform without replacement among eligible != 0."""
    el = np.ascontiguousarray(eligible.astype(np.uint8))
    taken = np.empty(n, dtype=np.uint8)
    out = np.empty(k, dtype=np.uint32)
    got = _load().gxs_sample(n, _ptr(el), k, (seed ^ SOURCE_TAG) & (2**64 - 1),
                             _ptr(taken), _ptr(out))
    if got != k:
        raise ValueError(f"only {got} of {k} eligible vertices found")
    return out


def sources_with_out_edges(n: int, src: np.ndarray, k: int, seed: int) -> np.ndarray:
    """Sources for multi-source runs: uniform over vertices of out-degree >= 1."""
    outdeg = np.bincount(src, minlength=n)
    return sample_vertices(n, outdeg > 0, k, seed)


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Open-loop Poisson arrival times in seconds: gaps -ln(1-u)/rate."""
    n_guess = int(rate_per_s * duration_s * 1.5) + 64
    u = stream_unit(seed ^ ARRIVE_TAG, 0, n_guess)
    t = np.cumsum(-np.log1p(-u) / rate_per_s)
    return t[t < duration_s]


def serve_stream(rate_per_s: float, duration_s: float, n_eligible, seed: int) -> dict:
    """The served query stream: Poisson arrival times; per query a graph
    uniform over len(n_eligible) graphs, a kind (0 = SSSP, 1 = PPR) with
    probability 1/2 each, and the index of its source among graph g's
    n_eligible[g] eligible sources (uniform). Each attribute has its own
    counter range of the seeded stream."""
    t = poisson_arrivals(rate_per_s, duration_s, seed)
    k = len(t)
    u_g = stream_unit(seed ^ SOURCE_TAG, 0, k)
    u_k = stream_unit(seed ^ SOURCE_TAG, 1 << 40, k)
    u_s = stream_unit(seed ^ SOURCE_TAG, 2 << 40, k)
    n_g = len(n_eligible)
    g = np.minimum((u_g * n_g).astype(np.int64), n_g - 1)
    cnt = np.asarray(n_eligible, dtype=np.int64)[g]
    pick = np.minimum((u_s * cnt).astype(np.int64), cnt - 1)
    return {"t": t, "graph": g, "kind": (u_k >= 0.5).astype(np.int64), "pick": pick}


def omp_threads() -> int:
    return int(_load().gxs_omp_threads())


@dataclasses.dataclass(frozen=True)
class Workload:
    """A seeded graph workload: its name says what it is and how big."""
    name: str
    kind: str            # "rmat", "er" or "clustered"
    scale: int           # log2 of the vertex count
    n_edges: int         # directed edges (ER: twice the pairs)
    seed: int
    w_lo: int = 0        # weights drawn in [w_lo, w_hi] when w_hi > 0
    w_hi: int = 0
    parts: int = 1       # contiguous dst-range partitions
    p_cross: float = 0.0 # clustered: fraction of pairs joining two blocks (blocks = parts)

    @property
    def n_vertices(self) -> int:
        return 1 << self.scale

    def edges(self):
        if self.kind == "rmat":
            src, dst = rmat(self.scale, self.n_edges, self.seed)
        elif self.kind == "er":
            src, dst = erdos_renyi(self.n_vertices, self.n_edges // 2, self.seed)
        elif self.kind == "clustered":
            src, dst = clustered(self.n_vertices, self.parts, self.n_edges // 2, self.p_cross, self.seed)
        else:
            raise ValueError(self.kind)
        w = weights(self.n_edges, self.w_lo, self.w_hi, self.seed) if self.w_hi else None
        return src, dst, w

    def scaled(self, scale: int) -> "Workload":
        """Same recipe at another size (edge factor kept)."""
        ef = self.n_edges // self.n_vertices
        return dataclasses.replace(self, name=f"{self.name}@s{scale}", scale=scale,
                                   n_edges=ef << scale)


# The five workloads: sizes, distributions and seeds.
SSSP_RMAT16 = Workload("sssp_rmat16", "rmat", 16, 1 << 20, 0x67700001, 1, 100)
PAGERANK_RMAT22 = Workload("pagerank_rmat22", "rmat", 22, 1 << 26, 0x67700002)
CC_ER24_P8 = Workload("cc_er24_8parts", "er", 24, 1 << 28, 0x67700003, parts=8)
# the same size, but 8 communities on the 8 partitions with one pair in
# 100,000 crossing between them, weighted: the graph on which sync skipping
# triggers (SSSP, as in the paper's skipping experiment)
SSSP_CLUSTERED24_P8 = Workload("sssp_clustered24_8parts", "clustered", 24, 1 << 28, 0x67700007, 1, 100, parts=8,
                               p_cross=1e-5)
MSSSP_RMAT24 = Workload("msssp64_rmat24", "rmat", 24, 1 << 28, 0x67700004, 1, 255)
# the SSSP recipe at the PageRank graph's size: where a pull sweep costs
# about a millisecond and the sparse supersteps are worth pushing
SSSP_RMAT22 = Workload("sssp_rmat22", "rmat", 22, 1 << 26, 0x67700006, 1, 100)
SERVE_SEED = 0x67700005
# served graphs: R-MAT scales 18/20/22/24, edge factor 16, w ~ U{1..255};
# seeds 0x67700018, 0x67700020, 0x67700022, 0x67700024 (the scale in hex digits)
SERVE_GRAPHS = tuple(Workload(f"serve_rmat{s}", "rmat", s, 16 << s, 0x67700000 + int(str(s), 16), 1, 255)
                     for s in (18, 20, 22, 24))
SERVE_RATE = 2000.0     # queries per second, open-loop Poisson
SERVE_SECONDS = 60.0
SERVE_DAMPING = 0.85
SERVE_ITERS = 20

WORKLOADS = {w.name: w for w in (SSSP_RMAT16, PAGERANK_RMAT22, CC_ER24_P8, MSSSP_RMAT24)}
