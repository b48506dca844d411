"""GPU parity of the affine-gap model (trioseq_plan_affine, affine.cu) against the oracle.

Natural gap costs (the build's reading of the paper's future work, Sec. VI): every score must
equal oracle.align_affine exactly, on all shapes up to 4^3, ragged and related batches under the
DNA and protein schemes with several openings, and a device-resident batch run repeatedly. With
gap_open = 0 the affine plan must reproduce the linear plan's scores. Traceback is not offered
for this model (ENOTIMPL), and only the global type is (EINVAL otherwise).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(1003)


def _strs(trips, sc):
    return [[synth.to_str(s, sc.alphabet) for s in t] for t in trips]


def _rand(rng, shapes, K):
    return [tuple(rng.integers(0, K, size=n).astype(np.uint8) for n in s) for s in shapes]


def _check(sc, gap_open, trips):
    plan = B.trioseq_plan_affine(sc.alphabet, sc.sub, sc.gap, gap_open)
    try:
        got = B.trioseq_align_batch(plan, _strs(trips, sc)).tolist()
    finally:
        B.trioseq_plan_destroy(plan)
    want = [oracle.align_affine(*t, sc.sub, sc.gap, gap_open) for t in trips]
    bad = [(i, got[i], want[i]) for i in range(len(trips)) if got[i] != want[i]]
    assert not bad, bad[:5]


@pytest.mark.parametrize("gap_open", [0, -1, -5])
def test_affine_all_tiny_shapes(gap_open):
    rng = np.random.default_rng(71)
    _check(DNA, gap_open, _rand(rng, itertools.product(range(5), repeat=3), 4))


@pytest.mark.parametrize("sc,gap_open", [(DNA, -3), (PROT, -8)], ids=["dna", "protein"])
def test_affine_ragged_shapes(sc, gap_open):
    rng = np.random.default_rng(72)
    shapes = [(37, 70, 55), (90, 12, 64), (0, 60, 61), (45, 0, 33), (50, 50, 0), (120, 3, 97),
              (1, 1, 1), (64, 65, 63)]
    _check(sc, gap_open, _rand(rng, shapes, len(sc.alphabet)))


def test_affine_related_batch():
    w = synth.config2(seed=73, n=48, lo=20, hi=90)
    _check(w.scoring, -4, w.triplets)


def test_affine_zero_opening_equals_linear_plan():
    w = synth.config2(seed=74, n=32, lo=10, hi=120)
    strs = _strs(w.triplets, w.scoring)
    aff = B.trioseq_plan_affine(w.scoring.alphabet, w.scoring.sub, w.scoring.gap, 0)
    lin = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    try:
        assert B.trioseq_align_batch(aff, strs).tolist() == B.trioseq_align_batch(lin, strs).tolist()
    finally:
        B.trioseq_plan_destroy(aff)
        B.trioseq_plan_destroy(lin)


def test_affine_resident_batch_repeats_and_limits():
    w = synth.config2(seed=75, n=20, lo=30, hi=80)
    strs = _strs(w.triplets, w.scoring)
    want = [oracle.align_affine(*t, w.scoring.sub, w.scoring.gap, -6) for t in w.triplets]
    plan = B.trioseq_plan_affine(w.scoring.alphabet, w.scoring.sub, w.scoring.gap, -6)
    try:
        bt = B.trioseq_batch_create(plan, strs)
        try:
            assert B.trioseq_batch_info(bt)["kernel"] == "affine_kernel"
            for _ in range(3):
                B.trioseq_batch_run(bt)
                assert B.trioseq_batch_scores(bt, len(strs)).tolist() == want
        finally:
            B.trioseq_batch_destroy(bt)
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_align_batch(plan, strs[:2], B.WITH_TRACEBACK)
        assert e.value.status == B.ENOTIMPL
    finally:
        B.trioseq_plan_destroy(plan)
    for flags, go in ((B.LOCAL, -2), (B.GLOBAL, 1)):
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_plan_affine(DNA.alphabet, DNA.sub, DNA.gap, go, flags)
        assert e.value.status == B.EINVAL
