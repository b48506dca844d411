"""GPU parity of the packed int16x2 mode: two triplets per column task, one per 16-bit half.

Scores must be identical to the oracle and to the same batch run unpacked (TRIOSEQ_PACKED=0).
Cases: odd batch sizes (the leftover triplet pairs with itself), mixed column-grid classes,
empty sequences, every tile, values near the int16 bound with positive and with negative
sigma'', and the cases that must stay unpacked (traceback, one triplet, lengths past the bound).
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


def _plan(sc, packed=True, tile=None):
    saved = {k: os.environ.get(k) for k in ("TRIOSEQ_PACKED", "TRIOSEQ_SCORE_TILE")}
    if not packed:
        os.environ["TRIOSEQ_PACKED"] = "0"
    if tile:
        os.environ["TRIOSEQ_SCORE_TILE"] = tile
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


def rand_trip(rng, shape, K):
    return tuple(rng.integers(0, K, size=n).astype(np.uint8) for n in shape)


def run(plan, sc, trips):
    s = [strs(t, sc) for t in trips]
    bt = B.trioseq_batch_create(plan, s)
    try:
        B.trioseq_batch_run(bt)
        return B.trioseq_batch_scores(bt, len(s)).tolist(), B.trioseq_batch_info(bt)["packing"]
    finally:
        B.trioseq_batch_destroy(bt)


@pytest.mark.parametrize("tile", ["4x4", "4x8", "8x8"])
def test_packed_equals_oracle_and_unpacked(tile):
    rng = np.random.default_rng(31)
    shapes = [(37, 70, 130), (129, 33, 65), (0, 100, 100), (100, 0, 77), (64, 64, 0),
              (200, 1, 250), (5, 260, 3), (31, 32, 63), (33, 65, 129), (1, 1, 1), (0, 0, 0)]
    trips = [rand_trip(rng, sh, 4) for sh in shapes]  # 11 triplets: one pairs with itself
    want = oracle.align_many(trips, DNA.sub, DNA.gap).tolist()
    pk, up = _plan(DNA, True, tile), _plan(DNA, False, tile)
    try:
        got, packing = run(pk, DNA, trips)
        assert packing == 2 and got == want
        got_u, packing_u = run(up, DNA, trips)
        assert packing_u == 1 and got_u == want
    finally:
        B.trioseq_plan_destroy(pk)
        B.trioseq_plan_destroy(up)


def test_packed_related_batch_and_protein():
    w = synth.config2(seed=93, n=37, lo=60, hi=300)
    plan = _plan(DNA)
    try:
        got, packing = run(plan, DNA, w.triplets)
        assert packing == 2
        assert got == oracle.align_many(w.triplets, DNA.sub, DNA.gap).tolist()
    finally:
        B.trioseq_plan_destroy(plan)
    rng = np.random.default_rng(32)
    trips = [rand_trip(rng, tuple(rng.integers(20, 200, size=3)), 20) for _ in range(9)]
    plan = _plan(PROT)
    try:
        got, packing = run(plan, PROT, trips)
        assert packing == 2
        assert got == oracle.align_many(trips, PROT.sub, PROT.gap).tolist()
    finally:
        B.trioseq_plan_destroy(plan)


def test_near_the_int16_bound():
    # DNA: max |sigma''| = 6, so a pair grid of a+b+c = 2727 sits just under 2^14 / 6 - 3.
    rng = np.random.default_rng(33)
    x = rng.integers(0, 4, size=909).astype(np.uint8)
    y = x.copy()
    y[::7] = (y[::7] + 1) % 4
    trips = [(x, x, x), (x, y, x)]
    plan = _plan(DNA)
    try:
        got, packing = run(plan, DNA, trips)
        assert packing == 2
        assert got[0] == 3 * int(DNA.sub[x, x].sum())  # identical triplet, closed form
        glob = _plan(DNA, False)
        try:
            got_u, _ = run(glob, DNA, trips)
        finally:
            B.trioseq_plan_destroy(glob)
        assert got == got_u
    finally:
        B.trioseq_plan_destroy(plan)


def test_negative_sigma_values_near_the_bound():
    # sigma'' = sigma - 2*alpha is negative off the diagonal here (-10 + 2), so the shifted values
    # fall as well as rise; max |sigma''| = 8 allows a pair grid of a+b+c up to 2044.
    sub = np.full((4, 4), -10, dtype=np.int64)
    np.fill_diagonal(sub, 6)
    sc = synth.Scoring("ACGT", sub.astype(np.int32), -1, np.full(4, 0.25), "negative")
    rng = np.random.default_rng(34)
    trips = [rand_trip(rng, (120, 130, 110), 4) for _ in range(3)]
    trips.append(rand_trip(rng, (680, 680, 680), 4))
    trips.append(rand_trip(rng, (680, 675, 684), 4))
    plan = _plan(sc)
    up = _plan(sc, False)
    try:
        got, packing = run(plan, sc, trips)
        assert packing == 2
        got_u, _ = run(up, sc, trips)
        assert got == got_u
        assert got[:3] == oracle.align_many(trips[:3], sc.sub, sc.gap).tolist()
    finally:
        B.trioseq_plan_destroy(plan)
        B.trioseq_plan_destroy(up)


def test_cases_that_stay_unpacked():
    rng = np.random.default_rng(35)
    plan = _plan(DNA)
    try:
        one = [rand_trip(rng, (50, 60, 70), 4)]
        got, packing = run(plan, DNA, one)
        assert packing == 1 and got == oracle.align_many(one, DNA.sub, DNA.gap).tolist()
        # past the bound: a+b+c = 3 x 1000 with max |sigma''| = 6
        big = [rand_trip(rng, (1000, 1000, 1000), 4), rand_trip(rng, (10, 10, 10), 4)]
        s = [strs(t, DNA) for t in big]
        bt = B.trioseq_batch_create(plan, s)
        try:
            assert B.trioseq_batch_info(bt)["packing"] == 1
        finally:
            B.trioseq_batch_destroy(bt)
        two = [rand_trip(rng, (30, 40, 50), 4), rand_trip(rng, (35, 45, 55), 4)]
        bt = B.trioseq_batch_create(plan, [strs(t, DNA) for t in two], B.WITH_TRACEBACK)
        try:
            assert B.trioseq_batch_info(bt)["packing"] == 1
        finally:
            B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)


def test_autotune_with_packing():
    w = synth.config2(seed=94, n=24, lo=40, hi=160)
    s = [strs(t, DNA) for t in w.triplets]
    plan = _plan(DNA)
    try:
        choice = B.trioseq_plan_autotune(plan, s, B.SCORE_ONLY)
        assert choice["tile"] in [(8, 8), (4, 8), (4, 4)]
        got = B.trioseq_align_batch(plan, s).tolist()
        assert got == oracle.align_many(w.triplets, DNA.sub, DNA.gap).tolist()
    finally:
        B.trioseq_plan_destroy(plan)
