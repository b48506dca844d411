"""GPU parity of slab launches: one triplet's cube cut into slabs of slices, each launch seeded
from the plane of stored values the slab below left.

With traceback this is the linear-space traceback: a forward pass keeps one plane per slab
boundary and no codes, then each slab from the top down recomputes its codes from the plane
below it and the walk continues through it. Scores and alignments must be bit-identical to the
one-launch path and to the oracle, for every slab height (one slice, heights that do not divide
the cube, a height above the cube), every tile, empty sequences, and at full size.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(1003)


def _plan(sc, slices=None, budget_mb=None, tb_tile=None, tile=None):
    keys = ("TRIOSEQ_SLAB_SLICES", "TRIOSEQ_SLAB_BUDGET_MB", "TRIOSEQ_TB_TILE",
            "TRIOSEQ_SCORE_TILE")
    saved = {k: os.environ.get(k) for k in keys}
    for k, v in zip(keys, (slices, budget_mb, tb_tile, tile)):
        if v is not None:
            os.environ[k] = str(v)
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def strs(trip, sc):
    return [synth.to_str(s, sc.alphabet) for s in trip]


def rows_str(rows, sc):
    return tuple("".join("-" if v == 255 else sc.alphabet[v] for v in row) for row in rows)


def run_one(plan, sc, t, mode):
    bt = B.trioseq_batch_create(plan, [strs(t, sc)], mode)
    try:
        B.trioseq_batch_run(bt)
        score = int(B.trioseq_batch_scores(bt, 1)[0])
        rows = B.trioseq_batch_alignment(bt, 0) if mode == B.WITH_TRACEBACK else None
        info = B.trioseq_batch_info(bt)
        return score, rows, (info["slab_slices"], info["slabs"])
    finally:
        B.trioseq_batch_destroy(bt)


@pytest.mark.parametrize("slices", [1, 7, 64, 1000])
@pytest.mark.parametrize("tile", ["4x4", "4x8", "8x8", "8x4"])
def test_traceback_slabs_match_oracle(slices, tile):
    w = synth.config2(seed=95, n=1, lo=150, hi=150)
    t = w.triplets[0]
    want, rows = oracle.align(*t, DNA.sub, DNA.gap, traceback=True)
    plan = _plan(DNA, slices=slices, tb_tile=tile)
    try:
        score, got_rows, (sl, ns) = run_one(plan, DNA, t, B.WITH_TRACEBACK)
        a = len(t[0])
        assert sl == min(slices, a + 1) and ns == -(-(a + 1) // sl)
        assert score == want
        assert got_rows == rows_str(rows, DNA)
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("slices", [1, 5, 33])
def test_score_slabs_match_oracle(slices):
    rng = np.random.default_rng(41)
    trips = [tuple(rng.integers(0, 20, size=n).astype(np.uint8) for n in sh)
             for sh in ((90, 130, 70), (0, 50, 60), (40, 0, 0), (1, 1, 1))]
    plan = _plan(PROT, slices=slices)
    try:
        for t in trips:
            score, _, (sl, ns) = run_one(plan, PROT, t, B.SCORE_ONLY)
            assert score == oracle.align(*t, PROT.sub, PROT.gap)
            assert sl == min(slices, len(t[0]) + 1)
    finally:
        B.trioseq_plan_destroy(plan)


def test_empty_and_degenerate_tracebacks():
    rng = np.random.default_rng(42)
    shapes = [(0, 0, 0), (0, 17, 9), (12, 0, 0), (1, 1, 1), (40, 2, 60)]
    plan = _plan(DNA, slices=3)
    try:
        for sh in shapes:
            t = tuple(rng.integers(0, 4, size=n).astype(np.uint8) for n in sh)
            want, rows = oracle.align(*t, DNA.sub, DNA.gap, traceback=True)
            score, got_rows, _ = run_one(plan, DNA, t, B.WITH_TRACEBACK)
            assert score == want and got_rows == rows_str(rows, DNA), sh
    finally:
        B.trioseq_plan_destroy(plan)


def test_budget_selects_slabs_and_config1_matches_one_launch():
    w = synth.config1()
    t = w.triplets[0]
    full = _plan(DNA)
    small = _plan(DNA, budget_mb=64)  # config 1 needs ~0.8 GB at once
    try:
        s_full, r_full, lay_full = run_one(full, DNA, t, B.WITH_TRACEBACK)
        s_slab, r_slab, lay_slab = run_one(small, DNA, t, B.WITH_TRACEBACK)
        assert lay_full == (0, 0) and lay_slab[1] > 1
        assert (s_slab, r_slab) == (s_full, r_full)
        # and through the one-call entry point
        got = B.trioseq_align_batch(small, [strs(t, DNA)], B.WITH_TRACEBACK)
        assert int(got[0]) == s_full and B.trioseq_traceback(small, 0) == r_full
    finally:
        B.trioseq_plan_destroy(full)
        B.trioseq_plan_destroy(small)


def test_large_protein_traceback_in_slabs():
    # n = 2000 protein: 8e9 cells, 4 GB of codes at once; in slabs of 250 slices.
    w = synth.config3(seed=43, L=2000)
    t = w.triplets[0]
    sc = w.scoring
    full = _plan(sc)
    slab = _plan(sc, slices=250)
    try:
        s_full, r_full, _ = run_one(full, sc, t, B.WITH_TRACEBACK)
        s_slab, r_slab, (sl, ns) = run_one(slab, sc, t, B.WITH_TRACEBACK)
        assert (sl, ns) == (250, -(-(len(t[0]) + 1) // 250))
        assert s_slab == s_full and r_slab == r_full
        enc = {ch: i for i, ch in enumerate(sc.alphabet)}
        rows = np.array([[255 if ch == "-" else enc[ch] for ch in row] for row in r_slab],
                        dtype=np.uint8)
        assert oracle.sp_score(rows, sc.sub, sc.gap) == s_slab  # the alignment scores its score
        for q in range(3):
            assert np.array_equal(rows[q][rows[q] != 255], t[q])
    finally:
        B.trioseq_plan_destroy(full)
        B.trioseq_plan_destroy(slab)
