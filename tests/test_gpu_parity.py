"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit for bit.

Scores are int32 and must be identical; alignments must be identical rows (the tie-break makes
the optimal alignment unique). Cases span several column blocks and ragged tails, empty and
degenerate sequences, both scoring schemes, all tile variants, score-only and traceback modes,
single triplets and mixed batches, and the full-size workloads (sampled where the oracle is too
slow to cover everything).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(1003)


def _plan(sc, tile=None, tb_tile=None):
    old = {}
    for k, v in (("TRIOSEQ_SCORE_TILE", tile), ("TRIOSEQ_TB_TILE", tb_tile)):
        old[k] = os.environ.get(k)
        if v:
            os.environ[k] = v
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.fixture(scope="module")
def dna_plan():
    p = _plan(DNA)
    yield p
    B.trioseq_plan_destroy(p)


@pytest.fixture(scope="module")
def prot_plan():
    p = _plan(PROT)
    yield p
    B.trioseq_plan_destroy(p)


def strs(trip, sc):
    return [synth.to_str(s, sc.alphabet) for s in trip]


def oracle_rows_str(rows, sc):
    return tuple("".join("-" if v == 255 else sc.alphabet[v] for v in row) for row in rows)


def check_batch(plan, sc, triplets, traceback):
    mode = B.WITH_TRACEBACK if traceback else B.SCORE_ONLY
    got = B.trioseq_align_batch(plan, [strs(t, sc) for t in triplets], mode)
    for i, t in enumerate(triplets):
        if traceback:
            want, rows = oracle.align(*t, sc.sub, sc.gap, traceback=True)
            assert int(got[i]) == want, (i, [len(x) for x in t])
            assert B.trioseq_traceback(plan, i) == oracle_rows_str(rows, sc), i
        else:
            want = oracle.align(*t, sc.sub, sc.gap)
            assert int(got[i]) == want, (i, [len(x) for x in t])
    return got


def rand_trip(rng, shape, K):
    return tuple(rng.integers(0, K, size=n).astype(np.uint8) for n in shape)


def test_all_tiny_shapes_one_batch(dna_plan):
    rng = np.random.default_rng(1)
    trips = [rand_trip(rng, s, 4) for s in itertools.product(range(6), repeat=3)]
    check_batch(dna_plan, DNA, trips, traceback=True)
    check_batch(dna_plan, DNA, trips, traceback=False)


@pytest.mark.parametrize("tile", ["4x4", "4x8", "8x8", "8x4"])
def test_ragged_multi_block_all_tiles(tile):
    rng = np.random.default_rng(2)
    shapes = [(37, 70, 130), (129, 33, 65), (0, 100, 100), (100, 0, 77), (64, 64, 0),
              (200, 1, 250), (5, 260, 3), (31, 32, 63), (33, 65, 129)]
    trips = [rand_trip(rng, s, 4) for s in shapes]
    plan = _plan(DNA, tile=None if tile == "8x4" else tile, tb_tile=tile)  # 8x4: traceback only
    try:
        check_batch(plan, DNA, trips, traceback=False)
        check_batch(plan, DNA, trips, traceback=True)
    finally:
        B.trioseq_plan_destroy(plan)


def test_protein_ragged(prot_plan):
    rng = np.random.default_rng(3)
    shapes = [(50, 90, 70), (130, 20, 140), (1, 1, 1), (0, 0, 9), (17, 0, 0), (0, 0, 0)]
    trips = [rand_trip(rng, s, 20) for s in shapes]
    check_batch(prot_plan, PROT, trips, traceback=True)
    check_batch(prot_plan, PROT, trips, traceback=False)


def test_config0_dna_128_exact(dna_plan):
    w = synth.config0()
    check_batch(dna_plan, DNA, w.triplets, traceback=True)


def test_related_mixed_batch(dna_plan):
    w = synth.config2(seed=77, n=48, lo=20, hi=140)
    check_batch(dna_plan, DNA, w.triplets, traceback=False)
    check_batch(dna_plan, DNA, w.triplets[:12], traceback=True)


def test_identical_and_permutations(prot_plan):
    rng = np.random.default_rng(4)
    x = rng.integers(0, 20, size=300).astype(np.uint8)
    got = B.trioseq_align_batch(prot_plan, [strs((x, x, x), PROT)])
    assert int(got[0]) == 3 * int(PROT.sub[x, x].sum())
    t = rand_trip(rng, (90, 150, 120), 20)
    perms = [tuple(t[q] for q in p) for p in itertools.permutations(range(3))]
    got = B.trioseq_align_batch(prot_plan, [strs(p, PROT) for p in perms])
    assert len(set(got.tolist())) == 1
    assert int(got[0]) == oracle.align(*t, PROT.sub, PROT.gap)


def test_alone_equals_in_batch(dna_plan):
    w = synth.config2(seed=5, n=20, lo=30, hi=90)
    batch = B.trioseq_align_batch(dna_plan, [strs(t, DNA) for t in w.triplets])
    for i in (0, 7, 19):
        alone = B.trioseq_align_batch(dna_plan, [strs(w.triplets[i], DNA)])
        assert int(alone[0]) == int(batch[i])
    tb = B.trioseq_align_batch(dna_plan, [strs(t, DNA) for t in w.triplets], B.WITH_TRACEBACK)
    assert tb.tolist() == batch.tolist()


def test_device_resident_batch_repeatable(dna_plan):
    w = synth.config2(seed=6, n=16, lo=40, hi=100)
    bt = B.trioseq_batch_create(dna_plan, [strs(t, DNA) for t in w.triplets], B.WITH_TRACEBACK)
    try:
        outs = []
        for _ in range(3):
            B.trioseq_batch_run(bt)
            outs.append(B.trioseq_batch_scores(bt, 16).tolist())
        assert outs[0] == outs[1] == outs[2]
        want = oracle.align_many(w.triplets, DNA.sub, DNA.gap).tolist()
        assert outs[0] == want
        for i in (0, 15):
            _, rows = oracle.align(*w.triplets[i], DNA.sub, DNA.gap, traceback=True)
            assert B.trioseq_batch_alignment(bt, i) == oracle_rows_str(rows, DNA)
        info = B.trioseq_batch_info(bt)
        assert info["n"] == 16 and info["cells"] == w.cells
    finally:
        B.trioseq_batch_destroy(bt)


def test_invalid_inputs(dna_plan):
    with pytest.raises(B.TrioseqError) as e:
        B.trioseq_align_batch(dna_plan, [("ACGX", "A", "C")])
    assert e.value.status == B.EINVAL
    with pytest.raises(B.TrioseqError):
        B.trioseq_plan("ACGT", np.array([[1, 2, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1]]),
                       -1)
    with pytest.raises(B.TrioseqError):
        B.trioseq_plan("AC", np.eye(2), 3)  # gap > 0
    B.trioseq_align_batch(dna_plan, [("ACG", "AC", "A")], B.WITH_TRACEBACK)
    with pytest.raises(B.TrioseqError):
        B.trioseq_traceback(dna_plan, 0, cap=2)  # alignment needs 3 columns


# ---- full-size workloads ----------------------------------------------------------------------

def test_config1_dna_1000_traceback_exact(dna_plan):
    w = synth.config1()
    check_batch(dna_plan, DNA, w.triplets, traceback=True)


def test_config2_batch_4096_sampled():
    w = synth.config2()
    plan = _plan(DNA)
    try:
        got = B.trioseq_align_batch(plan, [strs(t, DNA) for t in w.triplets])
        rng = np.random.default_rng(11)
        idx = sorted(set(rng.choice(len(w.triplets), size=10, replace=False).tolist()) | {0, 4095})
        want = oracle.align_many([w.triplets[i] for i in idx], DNA.sub, DNA.gap)
        assert [int(got[i]) for i in idx] == want.tolist()
    finally:
        B.trioseq_plan_destroy(plan)


def test_config2_batch_4096_traceback():
    """The 4096-triplet batch with traceback: every score equals the score-only run's, every
    alignment re-scores to its score and strips to its input triplet, and sampled alignments
    equal the oracle's."""
    w = synth.config2()
    sc = w.scoring
    plan = _plan(DNA)
    try:
        trip_strs = [strs(t, DNA) for t in w.triplets]
        score_only = B.trioseq_align_batch(plan, trip_strs)
        got = B.trioseq_align_batch(plan, trip_strs, B.WITH_TRACEBACK)
        assert got.tolist() == score_only.tolist()
        lut = np.full(256, 255, dtype=np.uint8)
        for code, ch in enumerate(sc.alphabet):
            lut[ord(ch)] = code
        for i, t in enumerate(w.triplets):
            rows = B.trioseq_traceback(plan, i)
            codes = np.stack([lut[np.frombuffer(r.encode(), dtype=np.uint8)] for r in rows])
            assert oracle.sp_score(codes, sc.sub, sc.gap) == int(got[i]), i
            for q in range(3):
                assert np.array_equal(codes[q][codes[q] != 255], t[q]), (i, q)
            assert not (codes == 255).all(axis=0).any(), i  # no all-gap column
        rng = np.random.default_rng(12)
        idx = sorted(set(rng.choice(len(w.triplets), size=8, replace=False).tolist()) | {0, 4095})
        for i in idx:
            score, rows = oracle.align(*w.triplets[i], sc.sub, sc.gap, traceback=True)
            assert int(got[i]) == score, i
            assert B.trioseq_traceback(plan, i) == oracle_rows_str(rows, sc), i
    finally:
        B.trioseq_plan_destroy(plan)


def test_config3_protein_4000_properties(prot_plan):
    w = synth.config3()
    t = w.triplets[0]
    sc = w.scoring
    plan = _plan(sc)
    try:
        got = B.trioseq_align_batch(plan, [strs(t, sc), strs((t[2], t[0], t[1]), sc)])
        assert int(got[0]) == int(got[1])  # permutation invariance at full size
        nw = [oracle.nw2(t[p], t[q], sc.sub, sc.gap) for p, q in ((0, 1), (0, 2), (1, 2))]
        assert int(got[0]) <= sum(nw)  # Carrillo-Lipman style upper bound
        # a smaller protein triplet of the same recipe, exact against the oracle
        w2 = synth.config3(seed=31, L=160)
        check_batch(plan, sc, w2.triplets, traceback=False)
    finally:
        B.trioseq_plan_destroy(plan)


def test_autotune_picks_a_variant_and_keeps_results(dna_plan):
    w = synth.config2(seed=88, n=24, lo=40, hi=160)
    strs = [strs_ for strs_ in ([synth.to_str(s, DNA.alphabet) for s in t] for t in w.triplets)]
    plan = _plan(DNA)
    try:
        before = B.trioseq_align_batch(plan, strs).tolist()
        choice = B.trioseq_plan_autotune(plan, strs, B.SCORE_ONLY)
        assert choice["tile"] in [(8, 8), (4, 8), (4, 4)] and choice["ti"] in (4, 8, 16, 32)
        bt = B.trioseq_batch_create(plan, strs)
        try:
            assert B.trioseq_batch_info(bt)["tile"] == choice["tile"]  # the cached choice is used
        finally:
            B.trioseq_batch_destroy(bt)
        assert B.trioseq_align_batch(plan, strs).tolist() == before
        assert before == oracle.align_many(w.triplets, DNA.sub, DNA.gap).tolist()
        choice_tb = B.trioseq_plan_autotune(plan, strs[:4], B.WITH_TRACEBACK)
        assert choice_tb["tile"] in [(8, 8), (4, 8), (4, 4), (8, 4)]  # 8x4: traceback only
        got = B.trioseq_align_batch(plan, strs[:4], B.WITH_TRACEBACK)
        for i in range(4):
            want, rows = oracle.align(*w.triplets[i], DNA.sub, DNA.gap, traceback=True)
            assert int(got[i]) == want
            assert B.trioseq_traceback(plan, i) == oracle_rows_str(rows, DNA)
    finally:
        B.trioseq_plan_destroy(plan)


def test_batch_run_graph_replay_matches_plain_launches():
    w = synth.config2(seed=91, n=10, lo=30, hi=120)
    strs_ = [strs(t, DNA) for t in w.triplets]
    os.environ["TRIOSEQ_GRAPHS"] = "0"
    try:
        plain_plan = _plan(DNA)
    finally:
        os.environ.pop("TRIOSEQ_GRAPHS")
    graph_plan = _plan(DNA)
    want = oracle.align_many(w.triplets, DNA.sub, DNA.gap).tolist()
    try:
        for plan in (plain_plan, graph_plan):
            bt = B.trioseq_batch_create(plan, strs_, B.WITH_TRACEBACK)
            try:
                for profile in (False, True, False):
                    B.trioseq_batch_profile(bt, profile)
                    for _ in range(2):
                        B.trioseq_batch_run(bt)
                        assert B.trioseq_batch_scores(bt, len(strs_)).tolist() == want
                    if profile:
                        ms = B.trioseq_batch_timing(bt)
                        assert ms[0] > 0 and ms[1] > 0
                _, rows = oracle.align(*w.triplets[3], DNA.sub, DNA.gap, traceback=True)
                assert B.trioseq_batch_alignment(bt, 3) == oracle_rows_str(rows, DNA)
            finally:
                B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plain_plan)
        B.trioseq_plan_destroy(graph_plan)
