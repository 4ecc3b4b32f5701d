"""Pins of the oracle's correctly rounded sum, the WCC-hat estimator, the
mean-field community score and the exact WCC against closed forms.

Paper passages: Methods > WCC (exact WCC(x,C)), Heuristic Counting of
Triangles (E[t(x,C)], E[t(x,V)], the upper bounds vt -> deg, WCC-hat(x,C),
WCC-hat(C), WCC-hat(P)).
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from paper_2210_03211_gb300 import workloads as W


def fsum_cases():
    rnd = random.Random(7)
    cases = [[], [1.0], [1e100, 1.0, -1e100], [0.1] * 10, [1.0, 1e-16, 1e-16],
             [2.0 ** 53, 1.0, 1.0], [5e-324, 5e-324, 1e-300],
             [1.0, 2.0 ** -53, 2.0 ** -106], [1.0, -2.0 ** -54, -2.0 ** -108]]
    for _ in range(40):
        k = rnd.randint(1, 400)
        cases.append([rnd.uniform(-1, 1) * 10.0 ** rnd.randint(-30, 30) for _ in range(k)])
    for _ in range(20):
        k = rnd.randint(1, 3000)
        cases.append([rnd.random() for _ in range(k)])
    return cases


@pytest.mark.parametrize("vals", fsum_cases())
def test_fsum_is_correctly_rounded(oracle_lib, vals):
    got = oracle_lib.fsum(vals)
    assert got == math.fsum(vals)
    if all(math.isfinite(v) for v in vals) and abs(sum(Fraction(v) for v in vals)) < 1e300:
        assert got == float(sum((Fraction(v) for v in vals), Fraction(0)))


@pytest.mark.parametrize("s", [2, 3, 4, 7, 20])
@pytest.mark.parametrize("cc", [1.0, 0.5, 0.125])
def test_estimator_on_isolated_clique(oracle_lib, s, cc):
    """A member of an isolated clique C = K_s: deg(x,C) = deg(x,V) = s-1, density
    p = 1, so WCC-hat(x,C) = C(s-1,2) / (C(s-1,2) cc) * (s-1)/(s-1) = 1/cc
    (0 when s = 2 since C(1,2) = 0).  The mean-field score sees the same
    members, so S = s/cc."""
    w = oracle_lib.wcchat_node(s - 1, s - 1, s, s * (s - 1) // 2, cc)
    S = oracle_lib.community_score(s, s * (s - 1) // 2, s * (s - 1), cc)
    if s == 2:
        assert w == 0.0 and S == 0.0
    else:
        assert w == pytest.approx(1.0 / cc, rel=1e-15)
        assert S == pytest.approx(s / cc, rel=1e-15)


def test_estimator_zero_cases(oracle_lib):
    assert oracle_lib.wcchat_node(3, 5, 1, 0, 0.5) == 0.0          # |C| < 2
    assert oracle_lib.wcchat_node(3, 5, 6, 9, 0.0) == 0.0          # E[t(x,V)] = 0
    assert oracle_lib.wcchat_node(1, 5, 6, 9, 0.5) == 0.0          # C(1,2) = 0
    assert oracle_lib.wcchat_node(3, 1, 6, 9, 0.5) == 0.0          # deg 1 -> E[t(x,V)] = 0
    assert oracle_lib.community_score(0, 0, 0, 0.5) == 0.0
    assert oracle_lib.community_score(1, 0, 7, 0.5) == 0.0
    assert oracle_lib.community_score(5, 2, 20, 0.5) == 0.0        # mean internal degree 0.8 < 1
    assert oracle_lib.community_score(5, 10, 25, 0.5) > 0.0


def test_estimator_against_exact_rationals(oracle_lib):
    """WCC-hat(x,C) written from the equation with exact fractions; the FP64
    value agrees to a few ulps (it rounds each of ~10 operations once)."""
    rnd = random.Random(3)
    for _ in range(500):
        n = rnd.randint(2, 3000)
        m = rnd.randint(0, n * (n - 1) // 2)
        d = rnd.randint(0, 5000)
        k = rnd.randint(0, min(d, n - 1))
        cc = rnd.random()
        p = Fraction(2 * m, n * (n - 1))
        b = lambda z: z * (z - 1) / 2 if z >= 1 else Fraction(0)
        ev = b(Fraction(d)) * Fraction(cc)
        ref = 0 if ev == 0 else b(Fraction(k)) * p / ev * Fraction(d) / ((n - 1) + (d - k))
        got = oracle_lib.wcchat_node(k, d, n, m, cc)
        assert got == pytest.approx(float(ref), rel=1e-13, abs=0)


def test_meanfield_score_equals_sum_on_uniform_communities(oracle_lib):
    """When every member has the same internal degree k and total degree d,
    the mean-field score S(n, m, vol) is exactly sum_x WCC-hat(x, C) (the
    homogeneity it assumes holds); only rounding differs."""
    for (s, extra) in [(4, 0), (6, 1), (10, 3), (25, 2)]:
        cc = 0.37
        # K_s with `extra` external edges per member: k = s-1, d = s-1+extra
        n, m = s, s * (s - 1) // 2
        vol = s * (s - 1 + extra)
        S = oracle_lib.community_score(n, m, vol, cc)
        tot = s * oracle_lib.wcchat_node(s - 1, s - 1 + extra, n, m, cc)
        assert S == pytest.approx(tot, rel=1e-14)
    # a cycle community C_s (k = 2 for everyone) inside a larger graph
    for s in (5, 9):
        for extra in (0, 3):
            S = oracle_lib.community_score(s, s, s * (2 + extra), 0.2)
            tot = s * oracle_lib.wcchat_node(2, 2 + extra, s, s, 0.2)
            assert S == pytest.approx(tot, rel=1e-14)


def test_gain_signs_on_cliques(oracle_lib):
    """Leaving an isolated clique lowers its score (S drops from s/cc to
    (s-3)/cc); a pendant node joining a clique lowers it too."""
    cc = 1.0
    for s in (4, 5, 8):
        m = s * (s - 1) // 2
        before = oracle_lib.community_score(s, m, s * (s - 1), cc)
        after_leave = oracle_lib.community_score(s - 1, m - (s - 1), s * (s - 1) - (s - 1), cc)
        assert after_leave - before < 0
        assert after_leave == pytest.approx((s - 3) / cc, rel=1e-14)
        # pendant node y (degree 1) attached to one member joins
        before_p = oracle_lib.community_score(s, m, s * (s - 1) + 1, cc)
        after_join = oracle_lib.community_score(s + 1, m + 1, s * (s - 1) + 2, cc)
        assert after_join - before_p < 0


def test_exact_wcc_and_estimator_agree_on_isolated_cliques(oracle_lib):
    """Exact WCC(x,C) = t(x,C)/t(x,V) * vt(x,V)/(|C\\{x}| + vt(x,V\\C)) = 1 for a
    member of an isolated clique (all its triangles and triangle partners are
    inside); WCC-hat(x,C) is 1 too when cc = 1 (every node of a disjoint union
    of cliques has CC = 1)."""
    pairs = W.clique(5, 0) + W.clique(6, 10)
    el = W.from_pairs(pairs)
    g = oracle_lib.OracleGraph(el.src, el.dst)
    assert g.cc == 1.0
    _, _, labels = g.csr()
    pos = {int(v): i for i, v in enumerate(labels)}
    for members in ([pos[i] for i in range(5)], [pos[10 + i] for i in range(6)]):
        s = len(members)
        for x in members:
            assert g.exact_wcc(x, members) == 1.0
            assert oracle_lib.wcchat_node(s - 1, s - 1, s, s * (s - 1) // 2, g.cc) == 1.0


def test_exact_wcc_on_bowtie(oracle_lib):
    """Bowtie (triangles {0,1,2} and {2,3,4}): node 2 in C = {0,1,2} has
    t(2,C) = 1, t(2,V) = 2, vt(2,V) = 4, |C\\{2}| = 2, vt(2,V\\C) = 2,
    so WCC = 1/2 * 4/4 = 1/2; node 0 has WCC = 1 * 2/2 = 1."""
    el = W.from_pairs([(0, 1), (0, 2), (1, 2), (2, 3), (2, 4), (3, 4)])
    g = oracle_lib.OracleGraph(el.src, el.dst)
    assert g.exact_wcc(2, [0, 1, 2]) == 0.5
    assert g.exact_wcc(0, [0, 1, 2]) == 1.0
