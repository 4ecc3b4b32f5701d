"""Pins of the oracle's F1-score for overlapping covers (Methods, Evaluation
Criteria: F1-Score for Overlapping Communities)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest


def a(*ids):
    return np.array(ids, dtype=np.int32)


def test_worked_example(oracle_lib):
    """C' = {1,2}, C = {1,2,3}: p = 1, r = 2/3, F1 = 2 (2/3) / (5/3) = 4/5."""
    f, best = oracle_lib.cover_f1([a(1, 2)], [a(1, 2, 3)])
    assert f == 0.8 and best.tolist() == [0]


def test_identical_covers_score_one_and_disjoint_zero(oracle_lib):
    cover = [a(1, 2, 3), a(3, 4), a(7, 8, 9, 10)]
    assert oracle_lib.cover_f1(cover, cover)[0] == 1.0
    f, best = oracle_lib.cover_f1([a(100, 101)], cover)
    assert f == 0.0 and best.tolist() == [-1]


def test_each_detected_community_takes_its_best_match(oracle_lib):
    """Mean over detected communities (not symmetric): {1,2} matches {1,2,3}
    (0.8), {7,8} matches {7,8,9,10} (2/3); mean (0.8 + 2/3) / 2."""
    f, best = oracle_lib.cover_f1([a(1, 2), a(7, 8)], [a(1, 2, 3), a(7, 8, 9, 10), a(2, 7)])
    assert best.tolist() == [0, 1]
    assert f == pytest.approx((0.8 + 2 / 3) / 2, rel=1e-15)
    # the other direction averages over the three reference communities
    g, _ = oracle_lib.cover_f1([a(1, 2, 3), a(7, 8, 9, 10), a(2, 7)], [a(1, 2), a(7, 8)])
    assert g != f


def test_equals_exact_rational_brute_force(oracle_lib):
    """Random small covers: each best F1 equals 2k/(|C'|+|C|) maximised by
    brute force in exact rationals (the printed formula, simplified), and the
    mean is within a rounding or two of the exact mean."""
    rng = np.random.default_rng(3)
    for trial in range(25):
        det = [np.unique(rng.integers(0, 30, rng.integers(1, 9))).astype(np.int32) for _ in range(rng.integers(1, 7))]
        ref = [np.unique(rng.integers(0, 30, rng.integers(1, 9))).astype(np.int32) for _ in range(rng.integers(1, 7))]
        f, best = oracle_lib.cover_f1(det, ref)
        total = Fraction(0)
        for i, c in enumerate(det):
            scores = [Fraction(2 * len(set(c) & set(r)), len(c) + len(r)) for r in ref]
            top = max(scores)
            total += top
            if top > 0:
                assert scores[best[i]] == top and best[i] == scores.index(top)
            else:
                assert best[i] == -1
        assert f == pytest.approx(float(total / len(det)), rel=4e-16, abs=0)


def test_invariant_under_reordering(oracle_lib):
    rng = np.random.default_rng(5)
    det = [np.unique(rng.integers(0, 50, 8)).astype(np.int32) for _ in range(6)]
    ref = [np.unique(rng.integers(0, 50, 10)).astype(np.int32) for _ in range(5)]
    f0, _ = oracle_lib.cover_f1(det, ref)
    for perm in itertools.islice(itertools.permutations(range(6)), 0, 720, 97):
        f1, _ = oracle_lib.cover_f1([rng.permutation(det[i]) for i in perm], ref[::-1])
        assert f1 == f0   # exact sum: the order of the terms does not matter
