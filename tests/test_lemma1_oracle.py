"""Pins for the block-size model (Lemma 1 and the pipeline-time equation).

The lemma's closed form is checked against brute force over the equation
itself: integer block counts s (b = d/s) and a dense grid of real b.
"""
import math

import numpy as np
import pytest

from oracle import lemma1 as L


def _brute_integer_s(k1, k2, k3, a, d, s_max=None):
    s_max = s_max or int(min(d, 4_000_000))
    s = np.arange(2, s_max + 1, dtype=np.float64)
    b = d / s
    tn, tc, tu = k1 * b, a + k2 * b, k3 * b
    t = tn + np.maximum(tn, tc) + (s - 2) * np.maximum(np.maximum(tn, tc), tu) + np.maximum(tc, tu) + tu
    i = int(np.argmin(t))
    return int(s[i]), float(t[i])


def _brute_real_b(k1, k2, k3, a, d):
    b = np.geomspace(1e-6 * d, d / 2, 400_001)
    s = d / b
    tn, tc, tu = k1 * b, a + k2 * b, k3 * b
    t = tn + np.maximum(tn, tc) + (s - 2) * np.maximum(np.maximum(tn, tc), tu) + np.maximum(tc, tu) + tu
    return float(t.min())


def test_t_total_hand_values():
    # s = 3 blocks of b = 10, k = (1, 2, 3), a = 5: T_n = 10, T_c = 25, T_u = 30
    # T = 10 + max(10,25) + 1*max(10,25,30) + max(25,30) + 30 = 10+25+30+30+30
    assert L.t_total(10, 3, 1, 2, 3, 5) == 125
    # no call cost, all k equal: T = k b (s + 2) = k (d + 2b)
    assert L.t_total(4, 5, 2, 2, 2, 0) == pytest.approx(2 * (20 + 8))


@pytest.mark.parametrize("algo", sorted(L.PAPER_COEFFS))
@pytest.mark.parametrize("d", [117_180_000, 1 << 26, 1 << 28])
def test_paper_coefficients_integer_rounding_is_brute_force_min(algo, d):
    k1, k2, k3, a = L.PAPER_COEFFS[algo]
    b, s, t = L.lemma1_integer(k1, k2, k3, a, d)
    s_bf, t_bf = _brute_integer_s(k1, k2, k3, a, d)
    assert t <= t_bf * (1 + 1e-12)
    assert abs(t - t_bf) <= 1e-9 * t_bf


def test_paper_pagerank_case():
    k1, k2, k3, a = L.PAPER_COEFFS["pagerank"]
    b, s, t, case = L.lemma1(k1, k2, k3, a, 1 << 26)
    assert case == "k2"               # k2 = 0.58 is the largest cost
    assert b == pytest.approx(math.sqrt(a * (1 << 26) / (k1 + k3)))
    assert s == pytest.approx(63.94, abs=0.01)


def _coeff_cases():
    rng = np.random.default_rng(42)
    out = []
    for _ in range(60):
        k = rng.uniform(0.01, 1.0, 3)
        a = float(10 ** rng.uniform(0, 5))
        d = float(10 ** rng.uniform(4, 8))
        out.append((float(k[0]), float(k[1]), float(k[2]), a, d))
    # forced cases: k1 dominant with a small call cost, k3 dominant, k2 dominant
    out += [(1.0, 0.1, 0.2, 10.0, 1e6), (0.2, 0.1, 1.0, 10.0, 1e6), (0.1, 1.0, 0.2, 10.0, 1e6),
            (1.0, 0.1, 0.2, 1e6, 1e6), (0.2, 0.1, 1.0, 1e6, 1e6)]
    return out


@pytest.mark.parametrize("k1,k2,k3,a,d", _coeff_cases())
def test_lemma_is_continuous_minimum(k1, k2, k3, a, d):
    b, s, t_min, case = L.lemma1(k1, k2, k3, a, d)
    if s < 2:
        pytest.skip("optimum below two blocks: the equation needs s >= 2")
    # the lemma's two formulas agree with each other
    assert L.t_total(b, d / b, k1, k2, k3, a) == pytest.approx(t_min, rel=1e-9)
    # and no block size on a dense grid does better
    t_grid = _brute_real_b(k1, k2, k3, a, d)
    assert t_min <= t_grid * (1 + 1e-9)
    assert t_grid <= t_min * (1 + 1e-4)


def test_all_three_cases_reached():
    cases = {L.lemma1(*c)[3] for c in _coeff_cases()}
    assert cases == {"k1", "k2", "k3"}
