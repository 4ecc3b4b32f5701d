"""The error bounds of the GPU's candidate screens, checked on the CPU.

Both screens only rule candidates out or pick a lone winner; the decision is
exact only if their bounds hold.  The device arithmetic is emulated here
operation by operation in numpy (float32 / float64 round to nearest, no fused
multiply-add; a fused one only rounds less) and compared with exact rational
values over random and adversarial inputs:

* mean-field departure: the FP32 closed form of the community score against
  the oracle's FP64 score, |S64 - S32| <= delta S32 with the delta the
  library ships (u32 = 2^-24, u64 = 2^-53, m the graph's edges):
      delta = 1.02 (21 u32 + u64 (200 + 8 m) + 2 u64) + 1e-9,
  the FP32 form having at most 15 roundings (relative error < 20 u32 + its
  own subtraction) and the FP64 form deviating from the exact score by at
  most u64 (m2 + 3 vol + 17);
* the paper's gain: the FP32 bracket X of a join or leave (community sums
  in FP64 stored as floats, neighbour corrections and the node's own term in
  FP32) against the oracle's gain -- the exactly summed, once rounded change
  of WCC-hat(P) -- |X - gain| <= E with the library's
      E = (1.5e-6 + (n + k + 64) 2.3e-16) M + (k + 16) 1.2e-7 p'/cc (|sum h| + g_x).
Paper passages: Heuristic Counting of Triangles (the estimator), the WCC-hat
sum equations, Node Changes (Joining / Leaving a Community).
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

U32 = 2.0 ** -24
U64 = 2.0 ** -53
f32 = np.float32
f64 = np.float64


def B(z):
    return z * (z - 1) / 2 if z >= 1 else Fr(0)


# ---------------------------------------------------------------------------
# mean-field: score32 emulated
# ---------------------------------------------------------------------------
def score32(n, m2, vol, cc32):
    if n < 2 or m2 <= n or vol <= n:
        return f32(0)
    a, b, c, e = f32(m2), f32(m2 - n), f32(n - 1), f32(vol - n)
    f = f32(f32(f32(n) * c) + f32(vol - m2))
    return f32(f32(f32(a * a) * b) / f32(f32(f32(c * e) * f) * cc32))


def score_exact(n, m2, vol, cc):
    if n < 2:
        return Fr(0)
    din, D, p = Fr(m2, n), Fr(vol, n), Fr(m2, n * (n - 1))
    ev = B(D) * cc
    if ev <= 0:
        return Fr(0)
    return n * (B(din) * p / ev) * (D / ((n - 1) + (D - din)))


def meanfield_cases(rng):
    out = []
    for _ in range(3000):
        n = int(rng.integers(2, 200000)) if rng.random() < 0.5 else int(rng.integers(2, 60))
        m2 = 2 * int(rng.integers(0, min(n * (n - 1), 2 ** 31 - 2) // 2 + 1))
        vol = m2 + int(rng.integers(0, 2 ** int(rng.integers(1, 31))))
        if vol >= 2 ** 32:
            continue
        out.append((n, m2, vol, float(rng.uniform(1e-4, 1.0))))
    # adversarial: cliques, m2 next to n, vol next to n, huge vol, tiny cc
    for n in (2, 3, 4, 5, 17, 1000, 65536):
        out += [(n, n * (n - 1), n * (n - 1) + 1, 1.0), (n, n + 2 - (n % 2), n + 3, 0.5),
                (n, n * (n - 1), 2 ** 31, 0.01), (n, min(n * (n - 1), 2 * n), n + 1, 1e-6)]
    return out


def test_meanfield_fp32_screen_bound(oracle_lib):
    rng = np.random.default_rng(17)
    checked = 0
    for n, m2, vol, cc in meanfield_cases(rng):
        s64 = oracle_lib.community_score(n, m2 // 2, vol, cc)
        s32 = float(score32(n, m2, vol, f32(cc)))
        ex = score_exact(n, m2, vol, Fr(cc))
        if ex == 0:
            assert s64 == 0.0
            continue
        exf = float(ex)
        # the FP64 estimator's own error
        assert abs(s64 - exf) <= U64 * (m2 + 3 * vol + 17) * exf * (1 + 1e-12), (n, m2, vol)
        if s32 == 0.0:   # only where the closed form's zero conditions hold
            assert m2 <= n or vol <= n
            continue
        assert abs(s32 - exf) <= 21 * U32 * exf, (n, m2, vol, cc)
        m = m2 // 2   # the community's edges: the tightest m the library could use
        delta = 1.02 * (21 * U32 + U64 * (200 + 8 * m) + 2 * U64) + 1e-9
        assert abs(s64 - s32) <= delta * s32, (n, m2, vol, cc)
        checked += 1
    assert checked > 2000


# ---------------------------------------------------------------------------
# the paper's gain: lit_screen emulated
# ---------------------------------------------------------------------------
def g32(k, d, nu):
    if k < 2 or d < 2:
        return f32(0)
    den = nu - 1 + d - k
    if den <= 0:
        return f32(0)
    kf, df = f32(k), f32(d)
    return f32(f32(f32(f32(0.5) * f32(kf * f32(kf - f32(1)))) * df) /
               f32(f32(f32(0.5) * f32(df * f32(df - f32(1)))) * f32(den)))


def h_join32(k, d, n):
    if d < 2 or k < 1:
        return f32(0)
    D, kf, df = f32(n + d - k), f32(k), f32(d)
    bk = f32(f32(0.5) * f32(kf * f32(kf - f32(1))))
    bd = f32(f32(0.5) * f32(df * f32(df - f32(1))))
    return f32(f32(df * f32(f32(kf * D) + bk)) / f32(bd * f32(D * f32(D - f32(1)))))


def h_leave32(k, d, n):
    if d < 2 or k < 2 or n < 3:
        return f32(0)
    D, kf, df = f32(n - 2 + d - k), f32(k), f32(d)
    bk1 = f32(f32(0.5) * f32(f32(kf - f32(1)) * f32(kf - f32(2))))
    bd = f32(f32(0.5) * f32(df * f32(df - f32(1))))
    return f32(-f32(f32(df * f32(bk1 + f32(f32(kf - f32(1)) * f32(D + f32(1))))) / f32(bd * f32(D * f32(D + f32(1))))))


def g64(k, d, nu):
    if k < 2 or d < 2:
        return 0.0
    den = nu - 1 + d - k
    if den <= 0:
        return 0.0
    bk = 0.5 * (float(k) * float(k - 1))
    bd = 0.5 * (float(d) * float(d - 1))
    return (bk * float(d)) / (bd * float(den))


def bracket(members, nbrs, x_k, x_d, own, cc, rng):
    """members: list of (k, d, count); nbrs: indices into members of x's
    neighbours in C (one member each, count >= 1).  The emulated
    k_lit_fsum + lit_screen: X and E (floats)."""
    n = sum(c for _, _, c in members)
    m2 = sum(k * c for k, _, c in members)
    F = []
    for nu in (n - 1, n, n + 1):   # FP64 sums, in numpy's pairwise order (the device sums in parallel)
        vals = np.repeat(np.array([g64(k, d, nu) for k, d, _ in members]), [c for _, _, c in members])
        F.append(f64(np.sum(rng.permutation(vals))))
    on = cc > 0 and n >= 1
    fstore = [f32(F[0]), f32(F[2]),
              f32(((m2 / (float(n) * float(n - 1))) / cc) * F[1]) if on and n >= 2 else f32(0),
              f32((1.0 / (float(n + 1) * float(n))) / cc) if on else f32(0),
              f32((1.0 / (float(n - 1) * float(n - 2))) / cc) if on and n - 1 >= 2 else f32(0)]
    k = x_k
    hs = f32(0)
    for i in rng.permutation(len(nbrs)):
        ky, dy, _ = members[nbrs[i]]
        hs = f32(hs + (h_leave32(ky, dy, n) if own else h_join32(ky, dy, n)))
    m2f = f32(m2)
    if not own:
        A = f32(f32(m2f + f32(2) * f32(k)) * fstore[3])
        gx = g32(k, x_d, n + 1)
        S1 = f32(f32(fstore[1] + hs) + gx)
        Sm = S1
        Eh = f32(hs + gx)
    else:
        A = f32(f32(m2f - f32(2) * f32(k)) * fstore[4])
        gx = g32(k, x_d, n - 1) if A != 0 else f32(0)
        S1 = f32(f32(fstore[0] - gx) + hs)
        Sm = f32(f32(fstore[0] + gx) - hs)
        Eh = f32(gx - hs)
    X = f32(f32(A * S1) - fstore[2])
    M = f32(f32(A * Sm) + fstore[2])
    E = f32(f32(f32(f32(1.5e-6) + f32(f32(f32(n + k) + f32(64)) * f32(2.3e-16))) * M) +
            f32(f32(f32(f32(k) + f32(16)) * f32(1.2e-7)) * f32(A * Eh)) + f32(1e-30))
    return float(X), float(E)


def oracle_gain(oracle_lib, members, nbrs, x_k, x_d, own, cc):
    """The oracle's gain: the estimator terms of C's members after and before
    the move and x's own term, each in FP64, summed exactly, rounded once."""
    n = sum(c for _, _, c in members)
    m2 = sum(k * c for k, _, c in members)
    m = m2 // 2
    nb = set(nbrs)
    if own:
        n1, m1 = n - 1, m - x_k
    else:
        n1, m1 = n + 1, m + x_k
    total = Fr(0)
    x_left = own   # a member of C that is x itself (own case): drop one copy of x's (k, d)
    for i, (k, d, c) in enumerate(members):
        copies = c
        if x_left and k == x_k and d == x_d:
            copies -= 1
            x_left = False
        adj = 1 if i in nb else 0   # the neighbour member (one copy) has deg(y,C) changed
        rest = copies - adj
        if adj:
            k1 = k - 1 if own else k + 1
            total += Fr(oracle_lib.wcchat_node(k1, d, n1, m1, cc)) - Fr(oracle_lib.wcchat_node(k, d, n, m, cc))
        if rest:
            total += rest * (Fr(oracle_lib.wcchat_node(k, d, n1, m1, cc)) - Fr(oracle_lib.wcchat_node(k, d, n, m, cc)))
    if own:
        total -= Fr(oracle_lib.wcchat_node(x_k, x_d, n, m, cc))
    else:
        total += Fr(oracle_lib.wcchat_node(x_k, x_d, n1, m1, cc))
    return float(total)


def random_case(rng, big=False):
    """A community as (k, d, count) groups with an even sum of internal
    degrees, a candidate node x and which members are x's neighbours."""
    while True:
        groups = int(rng.integers(1, 12))
        members = []
        for _ in range(groups):
            d = int(rng.integers(1, 40 if rng.random() < 0.7 else 5000))
            k = int(rng.integers(0, d + 1))
            c = int(rng.integers(1, 4 if not big else 20000))
            members.append([k, d, c])
        n = sum(c for _, _, c in members)
        if n < 1:
            continue
        for g in members:   # deg(y,C) <= n - 1
            g[0] = min(g[0], n - 1)
        if sum(k * c for k, _, c in members) % 2:
            members[0][0] = max(0, members[0][0] - 1) if members[0][0] > 0 else min(members[0][1], n - 1, 1)
            if sum(k * c for k, _, c in members) % 2:
                continue
        own = bool(rng.random() < 0.5) and n >= 1
        members = [tuple(g) for g in members]
        if own:
            # x is a member: a group with k >= (number of neighbours chosen)
            xi = int(rng.integers(0, len(members)))
            x_k, x_d = members[xi][0], members[xi][1]
            cand = [i for i, (k, d, c) in enumerate(members) if k >= 1 and i != xi]
            if len(cand) < x_k:
                continue
            nbrs = list(rng.choice(cand, size=x_k, replace=False)) if x_k else []
        else:
            x_d = int(rng.integers(1, 300))
            cand = [i for i, (k, d, c) in enumerate(members) if k <= d - 1]
            if not cand:
                continue
            x_k = int(rng.integers(1, min(len(cand), x_d) + 1))
            nbrs = list(rng.choice(cand, size=x_k, replace=False))
        return members, [int(i) for i in nbrs], x_k, x_d, own


@pytest.mark.parametrize("big", [False, True], ids=["small_communities", "communities_up_to_240k"])
def test_literal_fp32_bracket_bound(oracle_lib, big):
    rng = np.random.default_rng(23 + int(big))
    checked = 0
    for _ in range(1500 if not big else 300):
        members, nbrs, x_k, x_d, own = random_case(rng, big)
        cc = float(rng.choice([1.0, 0.5, 0.13, 1e-3, 3e-7]))
        want = oracle_gain(oracle_lib, members, nbrs, x_k, x_d, own, cc)
        X, E = bracket(members, nbrs, x_k, x_d, own, cc, rng)
        assert np.isfinite(X) and np.isfinite(E)
        assert abs(X - want) <= E, (members, nbrs, x_k, x_d, own, cc, X, E, want)
        checked += 1
    assert checked >= 300
