"""Block-size model of the pipeline shuffle (Section III-A, "Block Size Selection").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Notation follows the paper: a node holds d entities split evenly into s blocks
of b = d/s entities; k1, k2, k3 are the download, compute and upload cost per
entity and a is the fixed per-block cost of calling the device (T_call).

* ``t_total`` is the simplified pipeline-time equation (the one written with
  k1, k2, k3 and a), valid for s >= 2:
      T = k1 b + max(k1 b, a + k2 b) + (s-2) max(k1 b, a + k2 b, k3 b)
          + max(a + k2 b, k3 b) + k3 b
* ``lemma1`` is Lemma 1: with Q = sqrt(a d / (k1 + k3)),
      b_opt = a/(k1-k2)  if k1 is the largest k and a/(k1-k2) < Q,
              a/(k3-k2)  if k3 is the largest k and a/(k3-k2) < Q,
              Q          otherwise,
  and T_min = a(k1+k3)/(k1-k2) + k1 d, a(k1+k3)/(k3-k2) + k3 d, or
  k2 d + 2 sqrt((k1+k3) a d) in the same three cases. (The proof's closing
  discussion writes "k1 d" in its case (iii); the lemma's own statement says
  k3 d, and that is the reading taken here.)
* ``lemma1_integer`` applies the paper's rounding step: s and b must be
  integers, so floor/ceil of s_opt = d/b_opt and floor/ceil of b_opt are
  tried in the equation and the smallest estimate wins.
"""
from __future__ import annotations

import math


def t_total(b: float, s: float, k1: float, k2: float, k3: float, a: float) -> float:
    tn, tc, tu = k1 * b, a + k2 * b, k3 * b
    return tn + max(tn, tc) + (s - 2.0) * max(tn, tc, tu) + max(tc, tu) + tu


def lemma1(k1: float, k2: float, k3: float, a: float, d: float):
    """Continuous optimum: returns (b_opt, s_opt, t_min, case) with case in {"k1", "k3", "k2"}."""
    q = math.sqrt(a * d / (k1 + k3))
    kmax = max(k1, k2, k3)
    if k1 == kmax and k1 > k2 and a / (k1 - k2) < q:
        b = a / (k1 - k2)
        return b, d / b, a * (k1 + k3) / (k1 - k2) + k1 * d, "k1"
    if k3 == kmax and k3 > k2 and a / (k3 - k2) < q:
        b = a / (k3 - k2)
        return b, d / b, a * (k1 + k3) / (k3 - k2) + k3 * d, "k3"
    return q, d / q, k2 * d + 2.0 * math.sqrt((k1 + k3) * a * d), "k2"


def lemma1_integer(k1: float, k2: float, k3: float, a: float, d: int):
    """Rounded choice: returns (b, s, t_estimate) with integer s >= 2.

    Candidates: s in {floor(s_opt), ceil(s_opt)} with b = d/s, and
    b in {floor(b_opt), ceil(b_opt)} with s = d/b rounded up to whole blocks
    (the last block then holds the remainder; the equation still charges it
    as a full block). Each candidate is scored with ``t_total``.
    """
    b_opt, s_opt, _, _ = lemma1(k1, k2, k3, a, d)
    cands = []
    for s in {math.floor(s_opt), math.ceil(s_opt)}:
        s = max(2, min(int(s), int(d)))
        cands.append((d / s, s))
    for b in {math.floor(b_opt), math.ceil(b_opt)}:
        b = max(1, min(int(b), int(d) // 2 if d >= 2 else 1))
        cands.append((float(b), max(2, -(-int(d) // b))))
    best = min(cands, key=lambda bs: (t_total(bs[0], bs[1], k1, k2, k3, a), bs[1]))
    return best[0], best[1], t_total(best[0], best[1], k1, k2, k3, a)


# The paper's measured coefficients (Section V-B, "Block Size Selection"):
# (k1, k2, k3, a) for SSSP, PageRank, and a third set labelled SSSP again,
# read as the LP set since LP is the third algorithm plotted there.
PAPER_COEFFS = {
    "sssp": (0.03, 0.51, 0.09, 84671.0),
    "pagerank": (0.02, 0.58, 0.1, 1970.0),
    "lp": (0.003, 0.59, 0.006, 498.0),
}
