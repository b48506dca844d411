"""Pins of the oracle's semi-global and local scores (Sec. II "Semi-Global Alignments",
"Local Alignments"), each against something other than the variant code itself.

Definitions used as pins (alpha <= 0 throughout, as the library requires):
* Local: with v = 0 and zero axes, M[e] is the best score of an alignment path that starts at
  any cell s <= e and ends at e, or 0. The local score is therefore the best global SP score over
  all triplets of substrings S0[i0:i1], S1[j0:j1], S2[k0:k1] (empty substrings give 0).
* Semi-global: zero axes and v = -infinity make M[e] the best path score from a start cell on an
  axis (two of the three indices zero) to e; a path cannot gain while it runs along an axis,
  since every axis move costs 2*alpha <= 0. The score is the best such path ending on a last
  slice (i1 = a or j1 = b or k1 = c), i.e. the best global score over the substring triplets
  whose start has at least two zero indices and whose end has at least one full-length index.
The global score of a substring triplet comes from the global oracle (pinned by brute force in
test_oracle_pins.py) or, for the tiniest inputs, from the brute-force enumerator directly.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import synth
from tests.brute import brute_force

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(1003)


def rand_sub(rng, K, lo=-4, hi=5):
    m = rng.integers(lo, hi, size=(K, K))
    return np.triu(m) + np.triu(m, 1).T


def rseq(rng, n, K):
    return rng.integers(0, K, size=n).astype(np.uint8)


def _ranges(n):
    return [(i0, i1) for i0 in range(n + 1) for i1 in range(i0, n + 1)]


def local_by_substrings(t, sub, gap, glob=None):
    glob = glob or (lambda x, y, z: oracle.align(x, y, z, sub, gap))
    a, b, c = map(len, t)
    best = 0
    for (i0, i1), (j0, j1), (k0, k1) in itertools.product(_ranges(a), _ranges(b), _ranges(c)):
        best = max(best, glob(t[0][i0:i1], t[1][j0:j1], t[2][k0:k1]))
    return best


def semi_by_substrings(t, sub, gap, glob=None):
    glob = glob or (lambda x, y, z: oracle.align(x, y, z, sub, gap))
    a, b, c = map(len, t)
    best = None
    for i0, j0, k0 in itertools.product(range(a + 1), range(b + 1), range(c + 1)):
        if (i0 == 0) + (j0 == 0) + (k0 == 0) < 2:
            continue
        for i1, j1, k1 in itertools.product(range(i0, a + 1), range(j0, b + 1), range(k0, c + 1)):
            if not (i1 == a or j1 == b or k1 == c):
                continue
            v = glob(t[0][i0:i1], t[1][j0:j1], t[2][k0:k1])
            best = v if best is None else max(best, v)
    return best


@pytest.mark.parametrize("shape", list(itertools.product(range(3), repeat=3)))
def test_bruteforce_small_shapes(shape):
    rng = np.random.default_rng(sum(s * 7 ** q for q, s in enumerate(shape)))
    sub = rand_sub(rng, 3)
    gap = -int(rng.integers(0, 4))
    t = [rseq(rng, n, 3) for n in shape]
    glob = lambda x, y, z: brute_force(x, y, z, sub, gap)[0]  # noqa: E731
    assert oracle.align_type(*t, sub, gap, oracle.LOCAL) == local_by_substrings(t, sub, gap, glob)
    assert oracle.align_type(*t, sub, gap, oracle.SEMIGLOBAL) == semi_by_substrings(t, sub, gap,
                                                                                    glob)
    assert oracle.align_type(*t, sub, gap, oracle.GLOBAL) == glob(*t)


@pytest.mark.parametrize("seed", range(12))
def test_substring_definitions(seed):
    rng = np.random.default_rng(100 + seed)
    K = 4 if seed % 2 == 0 else 20
    sc = DNA if K == 4 else PROT
    shape = tuple(int(x) for x in rng.integers(0, 7, size=3))
    t = [rseq(rng, n, K) for n in shape]
    assert oracle.align_type(*t, sc.sub, sc.gap, oracle.LOCAL) == local_by_substrings(
        t, sc.sub, sc.gap)
    assert oracle.align_type(*t, sc.sub, sc.gap, oracle.SEMIGLOBAL) == semi_by_substrings(
        t, sc.sub, sc.gap)


@pytest.mark.parametrize("seed", range(8))
def test_ordering_and_invariances(seed):
    rng = np.random.default_rng(200 + seed)
    sc = DNA if seed % 2 == 0 else PROT
    K = sc.sub.shape[0]
    t = [rseq(rng, int(n), K) for n in rng.integers(0, 40, size=3)]
    g = oracle.align_type(*t, sc.sub, sc.gap, oracle.GLOBAL)
    s = oracle.align_type(*t, sc.sub, sc.gap, oracle.SEMIGLOBAL)
    l = oracle.align_type(*t, sc.sub, sc.gap, oracle.LOCAL)
    assert g == oracle.align(*t, sc.sub, sc.gap)
    assert l >= s >= g and l >= 0
    for p in itertools.permutations(range(3)):  # all three definitions are symmetric in S0..S2
        tp = [t[q] for q in p]
        assert oracle.align_type(*tp, sc.sub, sc.gap, oracle.SEMIGLOBAL) == s
        assert oracle.align_type(*tp, sc.sub, sc.gap, oracle.LOCAL) == l
    rev = [x[::-1].copy() for x in t]  # local (best substring triplet) is reversal invariant
    assert oracle.align_type(*rev, sc.sub, sc.gap, oracle.LOCAL) == l


@pytest.mark.parametrize("sc", [DNA, PROT], ids=["dna", "protein"])
def test_identical_triplet(sc):
    rng = np.random.default_rng(5)
    K = sc.sub.shape[0]
    x = rseq(rng, 60, K)
    want = 3 * int(sc.sub[x, x].sum())  # every diagonal entry is positive and dominates its row
    for kind in (oracle.GLOBAL, oracle.SEMIGLOBAL, oracle.LOCAL):
        assert oracle.align_type(x, x, x, sc.sub, sc.gap, kind) == want


def test_empty_and_planted_motif():
    for kind in (oracle.SEMIGLOBAL, oracle.LOCAL):
        assert oracle.align_type([], [], [], DNA.sub, DNA.gap, kind) == 0
    rng = np.random.default_rng(9)
    motif = rseq(rng, 25, 4)
    t = [np.concatenate([rseq(rng, n0, 4), motif, rseq(rng, n1, 4)])
         for n0, n1 in ((30, 5), (3, 40), (17, 17))]
    l = oracle.align_type(*t, DNA.sub, DNA.gap, oracle.LOCAL)
    assert l >= 3 * 2 * len(motif)  # the motif alone, matched in all three, scores 3*match*len
    # semi-global: S1 inside S0 with free leading/trailing parts of S0 (pairwise flavour with a
    # third sequence equal to S1) scores like aligning S1 to itself three ways.
    s0 = np.concatenate([rseq(rng, 20, 4), motif, rseq(rng, 20, 4)])
    s = oracle.align_type(s0, motif, motif, DNA.sub, DNA.gap, oracle.SEMIGLOBAL)
    assert s >= 3 * 2 * len(motif)


# ---- tracebacks of the semi-global and local types ----------------------------------------------

from tests.brute import GAP, brute_best_ending_at, brute_walk  # noqa: E402


def _strip(row):
    return np.array([r for r in row if r != GAP], dtype=np.uint8)


@pytest.mark.parametrize("shape", [s for s in itertools.product(range(4), repeat=3) if sum(s) <= 7])
def test_variant_traceback_bruteforce(shape):
    rng = np.random.default_rng(300 + sum(q * 5 ** n for n, q in enumerate(shape)))
    sub = rand_sub(rng, 3)
    gap = -int(rng.integers(0, 4))
    t = [rseq(rng, n, 3) for n in shape]
    for kind in (oracle.SEMIGLOBAL, oracle.LOCAL):
        score, rows, beg, end = oracle.align_type_tb(*t, sub, gap, kind)
        assert score == oracle.align_type(*t, sub, gap, kind)
        # the end cell is the first cell (i, j, k order) whose best ending score is the optimum
        cells = [(i, j, k) for i in range(shape[0] + 1) for j in range(shape[1] + 1)
                 for k in range(shape[2] + 1)
                 if kind == oracle.LOCAL or i == shape[0] or j == shape[1] or k == shape[2]]
        first = next(e for e in cells if brute_best_ending_at(*t, sub, gap, e, kind) == score)
        assert end == first
        # the path is the first optimal one in move priority order
        want_rows, want_beg = brute_walk(*t, sub, gap, end, kind, score)
        assert beg == want_beg
        assert rows.tolist() == [list(r) for r in want_rows]


@pytest.mark.parametrize("seed", range(10))
def test_variant_traceback_consistency(seed):
    rng = np.random.default_rng(400 + seed)
    sc = DNA if seed % 2 == 0 else PROT
    K = sc.sub.shape[0]
    t = [rseq(rng, int(n), K) for n in rng.integers(0, 60, size=3)]
    for kind in (oracle.SEMIGLOBAL, oracle.LOCAL):
        score, rows, beg, end = oracle.align_type_tb(*t, sc.sub, sc.gap, kind)
        assert score == oracle.align_type(*t, sc.sub, sc.gap, kind)
        assert all(b <= e for b, e in zip(beg, end))
        for q in range(3):
            assert np.array_equal(_strip(rows[q]), t[q][beg[q]:end[q]])
        assert not any(all(rows[q][c] == GAP for q in range(3)) for c in range(rows.shape[1]))
        assert oracle.sp_score(rows, sc.sub, sc.gap) == score  # the path scores the optimum
        if kind == oracle.SEMIGLOBAL:
            assert sum(b == 0 for b in beg) >= 2  # starts on an axis
            assert end[0] == len(t[0]) or end[1] == len(t[1]) or end[2] == len(t[2])
    g, grows, gb, ge = oracle.align_type_tb(*t, sc.sub, sc.gap, oracle.GLOBAL)
    want, wrows = oracle.align(*t, sc.sub, sc.gap, traceback=True)
    assert (g, gb, ge) == (want, (0, 0, 0), tuple(len(x) for x in t))
    assert np.array_equal(grows, wrows)
