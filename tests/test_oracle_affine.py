"""Pins of the affine-gap oracle (oracle_align_affine, oracle_gotoh2), on CPU.

The paper names affine gaps as future work (Sec. VI) and defines none. The reading implemented
is the sum-of-pairs score with natural gap costs (Altschul 1989) in Gotoh's affine form: each
pair's induced pairwise alignment (columns with a gap in both of its sequences deleted) scores
sigma per residue pair, alpha per residue against a gap, and gamma once per maximal run of gaps
in one sequence. These tests pin the oracle to things other than itself:

- brute force: every 3-way alignment of every shape up to 3 x 3 x 3 (and samples at 4 x 4 x 3),
  each scored by projecting it onto the three pairs explicitly (an independent Python scorer
  with no dynamic program), under random matrices, gaps and openings;
- gamma = 0 gives Eq. 1's score (the linear oracle, itself pinned by brute force);
- one empty sequence: the score is the textbook pairwise affine score of the other two plus, per
  non-empty one, one gap run against the empty sequence (alpha * length + gamma), a closed form
  that separates natural from quasi-natural gap costs;
- the textbook pairwise Gotoh score itself against brute-force pairwise enumeration;
- identical triplets align without gaps; invariance under permutation and reversal; the pairwise
  upper bound; the emitted alignment re-scores to the score and strips to the inputs.
"""
import itertools

import numpy as np
import pytest

import oracle

from .brute import MOVES


def pair_score(xr, yr, sub, gap, gap_open):
    """Affine score of one pairwise alignment (two rows, None = gap); columns with a gap in both
    rows are deleted first, then every maximal run of gaps in one row scores gap_open once."""
    total, last = 0, None  # last: which row the previous column had a gap in
    for x, y in zip(xr, yr):
        if x is None and y is None:
            continue
        if x is not None and y is not None:
            total += int(sub[x][y])
            last = None
        else:
            kind = 0 if x is None else 1
            total += gap + (0 if last == kind else gap_open)
            last = kind
    return total


def natural_sp(rows, sub, gap, gap_open):
    """Score of a 3-row alignment (None = gap): the sum of its three projections' scores."""
    return sum(pair_score(rows[p], rows[q], sub, gap, gap_open) for p, q in ((0, 1), (0, 2), (1, 2)))


def all_alignments(s0, s1, s2):
    """Every 3-way alignment (list of columns; None = gap), by plain recursion over the moves."""
    out = []

    def rec(i, j, k, cols):
        if i == 0 and j == 0 and k == 0:
            out.append(list(reversed(cols)))
            return
        for di, dj, dk in MOVES:
            if i < di or j < dj or k < dk:
                continue
            col = (s0[i - 1] if di else None, s1[j - 1] if dj else None, s2[k - 1] if dk else None)
            rec(i - di, j - dj, k - dk, cols + [col])

    rec(len(s0), len(s1), len(s2), [])
    return out


def brute_affine(s0, s1, s2, sub, gap, gap_open):
    best = None
    for cols in all_alignments(s0, s1, s2):
        rows = [[c[q] for c in cols] for q in range(3)]
        v = natural_sp(rows, sub, gap, gap_open)
        best = v if best is None else max(best, v)
    return best


def brute_pairwise(x, y, sub, gap, gap_open):
    """Best pairwise affine score by enumerating every pairwise alignment."""
    best = [None]

    def rec(i, j, cols):
        if i == 0 and j == 0:
            v = pair_score([c[0] for c in cols], [c[1] for c in cols], sub, gap, gap_open)
            best[0] = v if best[0] is None else max(best[0], v)
            return
        for di, dj in ((1, 1), (1, 0), (0, 1)):
            if i >= di and j >= dj:
                rec(i - di, j - dj, [(x[i - 1] if di else None, y[j - 1] if dj else None)] + cols)

    rec(len(x), len(y), [])
    return best[0]


def rand_scheme(rng, K):
    sub = rng.integers(-4, 3, size=(K, K))
    sub = np.triu(sub) + np.triu(sub, 1).T
    np.fill_diagonal(sub, rng.integers(2, 7, size=K))
    return sub.astype(np.int32), int(rng.integers(-4, 1)), int(rng.integers(-8, 1))


def test_brute_force_every_shape_up_to_3():
    rng = np.random.default_rng(3100)
    for shape in itertools.product(range(4), repeat=3):
        for _ in range(3):
            sub, gap, go = rand_scheme(rng, 3)
            t = [list(rng.integers(0, 3, size=n)) for n in shape]
            assert oracle.align_affine(*t, sub, gap, go) == brute_affine(*t, sub, gap, go), \
                (shape, t, gap, go)


def test_brute_force_samples_at_4x4x3():
    rng = np.random.default_rng(3101)
    for _ in range(3):
        sub, gap, go = rand_scheme(rng, 4)
        t = [list(rng.integers(0, 4, size=n)) for n in (4, 4, 3)]
        assert oracle.align_affine(*t, sub, gap, go) == brute_affine(*t, sub, gap, go)


def test_zero_opening_is_the_linear_model():
    rng = np.random.default_rng(3102)
    for _ in range(40):
        sub, gap, _ = rand_scheme(rng, 4)
        t = [rng.integers(0, 4, size=int(rng.integers(0, 25))).astype(np.uint8) for _ in range(3)]
        assert oracle.align_affine(*t, sub, gap, 0) == oracle.align(*t, sub, gap)


def test_pairwise_gotoh_against_brute_force():
    rng = np.random.default_rng(3103)
    for a, b in itertools.product(range(5), repeat=2):
        sub, gap, go = rand_scheme(rng, 3)
        x, y = list(rng.integers(0, 3, size=a)), list(rng.integers(0, 3, size=b))
        assert oracle.gotoh2(x, y, sub, gap, go) == brute_pairwise(x, y, sub, gap, go), (x, y)


def test_one_empty_sequence_reduces_to_pairwise_gotoh():
    # S2 empty: the pairs (0,2) and (1,2) induce a single gap run each (their all-gap columns
    # are deleted), so the score is gotoh(S0, S1) + alpha*(|S0|+|S1|) + gamma per non-empty one
    rng = np.random.default_rng(3104)
    for _ in range(60):
        sub, gap, go = rand_scheme(rng, 4)
        x = rng.integers(0, 4, size=int(rng.integers(0, 30))).astype(np.uint8)
        y = rng.integers(0, 4, size=int(rng.integers(0, 30))).astype(np.uint8)
        want = (oracle.gotoh2(x, y, sub, gap, go) + gap * (len(x) + len(y)) +
                go * ((len(x) > 0) + (len(y) > 0)))
        e = np.zeros(0, dtype=np.uint8)
        for order in ((x, y, e), (x, e, y), (e, x, y)):
            assert oracle.align_affine(*order, sub, gap, go) == want


def test_two_empty_and_all_empty():
    sub, gap, go = rand_scheme(np.random.default_rng(3105), 4)
    e = np.zeros(0, dtype=np.uint8)
    x = np.array([0, 3, 1, 2, 2], dtype=np.uint8)
    assert oracle.align_affine(x, e, e, sub, gap, go) == 2 * (gap * len(x) + go)
    assert oracle.align_affine(e, e, e, sub, gap, go) == 0


def test_identical_triplets_align_without_gaps():
    rng = np.random.default_rng(3106)
    for _ in range(20):
        sub, gap, go = rand_scheme(rng, 4)
        sub = np.where(np.eye(4, dtype=bool), sub, np.minimum(sub, 0)).astype(np.int32)
        x = rng.integers(0, 4, size=int(rng.integers(1, 40))).astype(np.uint8)
        assert oracle.align_affine(x, x, x, sub, gap, go) == 3 * int(sum(sub[v, v] for v in x))


def test_permutation_and_reversal_invariance():
    rng = np.random.default_rng(3107)
    for _ in range(15):
        sub, gap, go = rand_scheme(rng, 4)
        t = [rng.integers(0, 4, size=int(rng.integers(0, 18))).astype(np.uint8) for _ in range(3)]
        v = oracle.align_affine(*t, sub, gap, go)
        for perm in itertools.permutations(range(3)):
            assert oracle.align_affine(*[t[p] for p in perm], sub, gap, go) == v
        assert oracle.align_affine(*[s[::-1].copy() for s in t], sub, gap, go) == v


def test_pairwise_upper_bound():
    rng = np.random.default_rng(3108)
    for _ in range(20):
        sub, gap, go = rand_scheme(rng, 4)
        t = [rng.integers(0, 4, size=int(rng.integers(0, 25))).astype(np.uint8) for _ in range(3)]
        bound = sum(oracle.gotoh2(t[p], t[q], sub, gap, go) for p, q in ((0, 1), (0, 2), (1, 2)))
        assert oracle.align_affine(*t, sub, gap, go) <= bound


@pytest.mark.parametrize("seed", range(6))
def test_emitted_alignment_rescores_and_strips(seed):
    rng = np.random.default_rng(3110 + seed)
    sub, gap, go = rand_scheme(rng, 4)
    t = [rng.integers(0, 4, size=int(rng.integers(0, 30))).astype(np.uint8) for _ in range(3)]
    score, rows = oracle.align_affine(*t, sub, gap, go, traceback=True)
    assert score == oracle.align_affine(*t, sub, gap, go)
    cols = [[None if v == oracle.GAP else int(v) for v in r] for r in rows]
    assert natural_sp(cols, sub, gap, go) == score
    for q in range(3):
        assert [v for v in cols[q] if v is not None] == t[q].tolist()
    assert all(any(cols[q][c] is not None for q in range(3)) for c in range(rows.shape[1]))
