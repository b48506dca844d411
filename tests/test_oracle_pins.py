"""Pins for the CPU oracle against facts fixed by the paper's definitions and by mathematics.

Each check targets a plausible mistake: a dropped or mis-signed gap term, a wrong predecessor
index, a transposed operand, a broken tie-break or traceback. None of these tests uses a GPU.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import synth
from tests.brute import GAP, brute_force, column_score, count_alignments

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(7)


def rand_sub(rng, K, lo=-4, hi=5):
    """Random symmetric matrix (no structure assumed)."""
    m = rng.integers(lo, hi, size=(K, K)).astype(np.int32)
    return np.triu(m) + np.triu(m, 1).T


def rseq(rng, n, K):
    return rng.integers(0, K, size=n).astype(np.uint8)


def strip(row):
    return np.array([r for r in row if r != GAP], dtype=np.uint8)


# ---------------------------------------------------------------------------------------------
# 1. brute force over every alignment (Eq. 1 is exact: the DP optimum is the max over all paths)

def test_alignment_counts():
    # Known lattice-path counts with the 7 moves: (1,1,1) -> 13 (sanity of the enumerator).
    assert count_alignments(1, 1, 1) == 13
    assert count_alignments(2, 2, 2) == 409
    assert count_alignments(3, 3, 3) == 16081
    assert count_alignments(4, 4, 4) == 699121


@pytest.mark.parametrize("K,gap", [(3, -2), (4, -1), (2, -3)])
def test_bruteforce_all_small_shapes(K, gap):
    rng = np.random.default_rng(100 + K)
    sub = rand_sub(rng, K)
    for a, b, c in itertools.product(range(4), repeat=3):
        s = [rseq(rng, n, K) for n in (a, b, c)]
        want, want_rows = brute_force(*s, sub, gap)
        got, rows = oracle.align(*s, sub, gap, traceback=True)
        assert got == want, (a, b, c)
        assert rows.tolist() == want_rows, (a, b, c)


def test_bruteforce_444():
    rng = np.random.default_rng(5)
    sub = DNA.sub
    s = [rseq(rng, 4, 4) for _ in range(3)]
    want, want_rows = brute_force(*s, sub, DNA.gap)
    got, rows = oracle.align(*s, sub, DNA.gap, traceback=True)
    assert got == want
    assert rows.tolist() == want_rows


def test_bruteforce_ties_low_entropy():
    # Binary alphabet and all-equal scores produce many ties: exercises the tie-break order.
    sub = np.array([[1, 1], [1, 1]], dtype=np.int32)
    rng = np.random.default_rng(9)
    for shape in [(3, 2, 3), (2, 3, 3), (3, 3, 1), (1, 3, 3)]:
        s = [rseq(rng, n, 2) for n in shape]
        want, want_rows = brute_force(*s, sub, -1)
        got, rows = oracle.align(*s, sub, -1, traceback=True)
        assert got == want and rows.tolist() == want_rows


# ---------------------------------------------------------------------------------------------
# 2. golden hand-worked examples

def _load_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "hand_dna.tsv")
    cases = []
    for line in open(path):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.rstrip("\n").split("\t")
        seqs = ["" if x == "." else x for x in f[:3]]
        rows = f[4:7] if len(f) >= 7 else None
        cases.append((seqs, int(f[3]), rows))
    return cases


def _enc(s):
    return np.array(["ACGT".index(ch) for ch in s], dtype=np.uint8)


@pytest.mark.parametrize("case", _load_golden())
def test_golden_hand_examples(case):
    seqs, score, rows = case
    got, r = oracle.align(*[_enc(s) for s in seqs], DNA.sub, DNA.gap, traceback=True)
    assert got == score
    if rows is not None:
        txt = ["".join("-" if v == GAP else "ACGT"[v] for v in row) for row in r]
        assert txt == rows


# ---------------------------------------------------------------------------------------------
# 3. reductions to pairwise Needleman-Wunsch (global init and the 2-D face recurrences)

@pytest.mark.parametrize("seed", range(6))
def test_one_empty_reduces_to_pairwise(seed):
    rng = np.random.default_rng(seed)
    sc = DNA if seed % 2 == 0 else PROT
    a, b = rng.integers(0, 40, size=2)
    x, y = rseq(rng, a, sc.K), rseq(rng, b, sc.K)
    nw = oracle.nw2(x, y, sc.sub, sc.gap)
    want = nw + sc.gap * (len(x) + len(y))
    e = np.zeros(0, dtype=np.uint8)
    # the empty sequence in each of the three positions (faces i=0, j=0, k=0)
    assert oracle.align(x, y, e, sc.sub, sc.gap) == want
    assert oracle.align(x, e, y, sc.sub, sc.gap) == want
    assert oracle.align(e, x, y, sc.sub, sc.gap) == want


def test_two_and_three_empty():
    rng = np.random.default_rng(1)
    e = np.zeros(0, dtype=np.uint8)
    for n in (1, 5, 33):
        x = rseq(rng, n, 4)
        for g in (-1, -2, -7):
            assert oracle.align(x, e, e, DNA.sub, g) == 2 * g * n
            assert oracle.align(e, x, e, DNA.sub, g) == 2 * g * n
            assert oracle.align(e, e, x, DNA.sub, g) == 2 * g * n
    assert oracle.align(e, e, e, DNA.sub, -2) == 0


# ---------------------------------------------------------------------------------------------
# 4. closed form for identical triplets

@pytest.mark.parametrize("sc", [DNA, PROT], ids=["dna", "protein"])
def test_identical_triplet_closed_form(sc):
    # Valid when every off-diagonal entry is below the diagonal entries and alpha <= 0: the SP
    # score is the sum of the three induced pairwise scores, each maximised by identity.
    assert (sc.sub.diagonal()[:, None] > sc.sub - np.diag(np.full(sc.K, 10**6))).all()
    rng = np.random.default_rng(3)
    for n in (1, 7, 64, 150):
        x = rseq(rng, n, sc.K)
        want = 3 * int(sc.sub[x, x].sum())
        got, rows = oracle.align(x, x, x, sc.sub, sc.gap, traceback=True)
        assert got == want
        assert (rows == x[None, :]).all()
    x = rseq(rng, 100, 4)
    assert oracle.align(x, x, x, DNA.sub, DNA.gap) == 3 * 100 * 2


# ---------------------------------------------------------------------------------------------
# 5. symmetries

@pytest.mark.parametrize("seed", range(4))
def test_permutation_invariance(seed):
    rng = np.random.default_rng(10 + seed)
    sc = DNA if seed % 2 else PROT
    s = [rseq(rng, int(n), sc.K) for n in rng.integers(0, 30, size=3)]
    ref = oracle.align(*s, sc.sub, sc.gap)
    for p in itertools.permutations(range(3)):
        assert oracle.align(*[s[q] for q in p], sc.sub, sc.gap) == ref


@pytest.mark.parametrize("seed", range(4))
def test_reversal_invariance(seed):
    rng = np.random.default_rng(20 + seed)
    sc = DNA if seed % 2 else PROT
    s = [rseq(rng, int(n), sc.K) for n in rng.integers(0, 30, size=3)]
    assert oracle.align(*[x[::-1].copy() for x in s], sc.sub, sc.gap) == \
        oracle.align(*s, sc.sub, sc.gap)


# ---------------------------------------------------------------------------------------------
# 6. re-scoring of the emitted alignment, and its validity

@pytest.mark.parametrize("seed", range(6))
def test_rescoring_and_validity(seed):
    rng = np.random.default_rng(30 + seed)
    sc = DNA if seed % 2 else PROT
    s = [rseq(rng, int(n), sc.K) for n in rng.integers(0, 60, size=3)]
    score, rows = oracle.align(*s, sc.sub, sc.gap, traceback=True)
    assert oracle.sp_score(rows, sc.sub, sc.gap) == score
    # independent Python re-scoring with the column definition
    tot = sum(column_score(tuple(None if v == GAP else int(v) for v in rows[:, t]),
                           sc.sub, sc.gap) for t in range(rows.shape[1]))
    assert tot == score
    for q in range(3):
        assert np.array_equal(strip(rows[q]), s[q])
    assert not (rows == GAP).all(axis=0).any()


# ---------------------------------------------------------------------------------------------
# 7. Carrillo-Lipman style upper bound and induced pairwise bounds

def _induced(r1, r2):
    keep = ~((r1 == GAP) & (r2 == GAP))
    return r1[keep], r2[keep]


def _pair_score(r1, r2, sub, gap):
    s = 0
    for u, v in zip(r1, r2):
        if u == GAP and v == GAP:
            continue
        s += gap if (u == GAP or v == GAP) else int(sub[u][v])
    return s


@pytest.mark.parametrize("seed", range(5))
def test_pairwise_upper_bounds(seed):
    rng = np.random.default_rng(40 + seed)
    sc = DNA if seed % 2 else PROT
    s = [rseq(rng, int(n), sc.K) for n in rng.integers(1, 50, size=3)]
    score, rows = oracle.align(*s, sc.sub, sc.gap, traceback=True)
    nw = {(p, q): oracle.nw2(s[p], s[q], sc.sub, sc.gap) for p, q in [(0, 1), (0, 2), (1, 2)]}
    assert score <= sum(nw.values())
    tot = 0
    for (p, q), bound in nw.items():
        r1, r2 = _induced(rows[p], rows[q])
        ps = _pair_score(r1, r2, sc.sub, sc.gap)
        assert ps <= bound
        tot += ps
    assert tot == score  # SP = sum of the three induced pairwise scores


# ---------------------------------------------------------------------------------------------
# 8. super-additivity under concatenation

@pytest.mark.parametrize("seed", range(4))
def test_superadditivity(seed):
    rng = np.random.default_rng(50 + seed)
    sc = DNA if seed % 2 else PROT
    s1 = [rseq(rng, int(n), sc.K) for n in rng.integers(0, 25, size=3)]
    s2 = [rseq(rng, int(n), sc.K) for n in rng.integers(0, 25, size=3)]
    cat = [np.concatenate([u, v]) for u, v in zip(s1, s2)]
    assert oracle.align(*cat, sc.sub, sc.gap) >= \
        oracle.align(*s1, sc.sub, sc.gap) + oracle.align(*s2, sc.sub, sc.gap)


# ---------------------------------------------------------------------------------------------
# 9. the batch helper agrees with single calls

def test_align_many_matches_single():
    w = synth.config2(n=6, lo=10, hi=40)
    got = oracle.align_many(w.triplets, w.scoring.sub, w.scoring.gap)
    want = [oracle.align(*t, w.scoring.sub, w.scoring.gap) for t in w.triplets]
    assert got.tolist() == want


def test_align_many_threads_match_one_core():
    w = synth.config2(seed=12, n=40, lo=20, hi=60)
    one = oracle.align_many(w.triplets, DNA.sub, DNA.gap)
    many = oracle.align_many(w.triplets, DNA.sub, DNA.gap, threads=4)
    assert one.tolist() == many.tolist()
