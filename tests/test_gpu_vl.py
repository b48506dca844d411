"""GPU parity of the two-cells-per-register score kernel (wavefront_vl.cuh, tile 8x16) against the
CPU oracle, bit for bit.

The kernel holds two column halves of one lane tile as the 16-bit halves of each register, the
high half one slice behind, against a per-task base that moves as the values grow. Cases: every
shape up to 5^3, ragged multi-block shapes for DNA and protein (several column tasks, tails in
both halves, empty sequences), related batches, medium triplets whose values force many
rebases, and the full-size workloads against the int32 kernel, which is itself checked against
the oracle elsewhere.
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
# the instantiations: 8 x (8+8) cells per lane (32 x 128 tasks) and 8 x (4+4) (32 x 64 tasks)
# with the sigma''(y,z) tile in registers, and 8 x (8+8) with it in shared memory (2-warp CTAs,
# "8x16s", or 1-warp CTAs, "8x16t")
VL_TILES = ["8x16", "8x8v", "8x16s", "8x16t"]


def _plan(sc, tile="8x16"):
    old = os.environ.get("TRIOSEQ_SCORE_TILE")
    os.environ["TRIOSEQ_SCORE_TILE"] = tile
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
    finally:
        if old is None:
            os.environ.pop("TRIOSEQ_SCORE_TILE", None)
        else:
            os.environ["TRIOSEQ_SCORE_TILE"] = old


def strs(trip, sc):
    return [synth.to_str(s, sc.alphabet) for s in trip]


def rand_trip(rng, shape, K):
    return tuple(rng.integers(0, K, size=n).astype(np.uint8) for n in shape)


def check(plan, sc, trips):
    got = B.trioseq_align_batch(plan, [strs(t, sc) for t in trips])
    want = oracle.align_many(trips, sc.sub, sc.gap)
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("tile", VL_TILES)
def test_vl_is_selected_for_nonnegative_schemes(tile):
    plan = _plan(DNA, tile)
    try:
        bt = B.trioseq_batch_create(plan, [["ACGT" * 20, "ACG" * 20, "AGT" * 20]])
        try:
            info = B.trioseq_batch_info(bt)
            assert info["tile"] == ((8, 8) if tile == "8x8v" else (8, 16))
            assert info["tile_label"] == tile and info["kernel"].startswith("wavefront_vl_kernel")
            assert info["packing"] == 2
        finally:
            B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", VL_TILES)
def test_vl_all_tiny_shapes_one_batch(tile):
    rng = np.random.default_rng(51)
    trips = [rand_trip(rng, s, 4) for s in itertools.product(range(6), repeat=3)]
    plan = _plan(DNA, tile)
    try:
        check(plan, DNA, trips)
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", VL_TILES)
@pytest.mark.parametrize("sc", [DNA, PROT], ids=["dna", "protein"])
def test_vl_ragged_multi_block(sc, tile):
    rng = np.random.default_rng(52)
    shapes = [(37, 70, 130), (129, 33, 65), (0, 100, 100), (100, 0, 77), (64, 64, 0),
              (200, 1, 250), (5, 260, 3), (31, 32, 63), (33, 65, 129), (17, 127, 128),
              (40, 135, 257), (1, 1, 1), (0, 0, 0)]
    trips = [rand_trip(rng, s, len(sc.alphabet)) for s in shapes]
    plan = _plan(sc, tile)
    try:
        check(plan, sc, trips)
        for t in trips[:4]:  # alone as well as in the batch
            check(plan, sc, [t])
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", VL_TILES)
def test_vl_related_batch_and_rebasing(tile):
    w = synth.config2(seed=98, n=24, lo=40, hi=300)
    big = synth.config1(seed=99, L=600).triplets  # values grow past many rebase thresholds
    prot = synth.config3(seed=97, L=420)
    plan = _plan(DNA, tile)
    try:
        check(plan, DNA, w.triplets + big)
    finally:
        B.trioseq_plan_destroy(plan)
    plan = _plan(prot.scoring, tile)
    try:
        check(plan, prot.scoring, prot.triplets)
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", VL_TILES)
@pytest.mark.parametrize("which", ["config1", "config3"])
def test_vl_full_size_equals_int32(which, tile):
    w = synth.config1() if which == "config1" else synth.config3()
    s = [strs(t, w.scoring) for t in w.triplets]
    ref = _plan(w.scoring, "8x8")
    vl = _plan(w.scoring, tile)
    try:
        want = B.trioseq_align_batch(ref, s)
        got = B.trioseq_align_batch(vl, s)
        assert got.tolist() == want.tolist()
    finally:
        B.trioseq_plan_destroy(vl)
        B.trioseq_plan_destroy(ref)


def test_vl_unavailable_cases_fall_back_to_int32():
    """Schemes with a negative sigma'' and the semi-global type cannot take the two-per-register
    kernel: a plan with its tile forced runs them on the int32 8x8 kernel, exactly. Traceback
    keeps its own tile."""
    neg = np.full((4, 4), -10, dtype=np.int8)  # sigma'' = -10 + 4 < 0 off the diagonal
    np.fill_diagonal(neg, 2)
    neg_sc = type("Sc", (), {"alphabet": "ACGT", "sub": neg, "gap": -2})
    rng = np.random.default_rng(53)
    trips = [rand_trip(rng, s, 4) for s in ((40, 70, 150), (130, 33, 64))]
    plan = _plan(neg_sc)
    try:
        check(plan, neg_sc, trips)
        bt = B.trioseq_batch_create(plan, [strs(t, neg_sc) for t in trips])
        try:
            assert B.trioseq_batch_info(bt)["tile"] == (8, 8)
        finally:
            B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)
    old = os.environ.get("TRIOSEQ_SCORE_TILE")
    os.environ["TRIOSEQ_SCORE_TILE"] = "8x16"
    try:
        semi = B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap, B.SEMIGLOBAL)
    finally:
        if old is None:
            os.environ.pop("TRIOSEQ_SCORE_TILE", None)
        else:
            os.environ["TRIOSEQ_SCORE_TILE"] = old
    try:
        got = B.trioseq_align_batch(semi, [strs(t, DNA) for t in trips])
        want = [oracle.align_type(*t, DNA.sub, DNA.gap, oracle.SEMIGLOBAL) for t in trips]
        assert got.tolist() == want
    finally:
        B.trioseq_plan_destroy(semi)
    plan = _plan(DNA)
    try:
        t = tuple(np.array([DNA.alphabet.index(ch) for ch in x], dtype=np.uint8)
                  for x in ("ACGTTGCA", "ACGTGCA", "AGTTGCA"))
        got = B.trioseq_align_batch(plan, [strs(t, DNA)], B.WITH_TRACEBACK)
        score, rows = oracle.align(*t, DNA.sub, DNA.gap, traceback=True)
        assert int(got[0]) == score
    finally:
        B.trioseq_plan_destroy(plan)


def _semi_plan(sc, tile, flags=None):
    old = os.environ.get("TRIOSEQ_SCORE_TILE")
    os.environ["TRIOSEQ_SCORE_TILE"] = tile
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap,
                              B.SEMIGLOBAL if flags is None else flags)
    finally:
        if old is None:
            os.environ.pop("TRIOSEQ_SCORE_TILE", None)
        else:
            os.environ["TRIOSEQ_SCORE_TILE"] = old


@pytest.mark.parametrize("tile", ["8x16", "8x8v"])
@pytest.mark.parametrize("kind,flags", [(oracle.SEMIGLOBAL, B.SEMIGLOBAL), (oracle.LOCAL, B.LOCAL)],
                         ids=["semiglobal", "local"])
def test_vl_variant_types_exact(tile, kind, flags):
    """The semi-global type (Sec. II: zero axes, best cell on a last slice) and the local type
    (zero axes, v = 0, best cell of the cube) on the two-cells-per-register kernel: every shape up
    to 4^3, ragged multi-block DNA and protein shapes (empty sequences included), related
    triplets whose values force rebases; exact against oracle.align_type. The batch must run on
    the two-per-register kernel."""
    rng = np.random.default_rng(81)
    cases = [(DNA, [rand_trip(rng, s, 4) for s in itertools.product(range(5), repeat=3)]),
             (DNA, [rand_trip(rng, s, 4) for s in ((37, 70, 130), (129, 33, 65), (0, 100, 100),
                                                  (100, 0, 77), (64, 64, 0), (200, 1, 250),
                                                  (33, 65, 129), (40, 135, 257))]),
             (PROT, [rand_trip(rng, s, 20) for s in ((90, 140, 260), (31, 32, 63), (5, 260, 3))]),
             (DNA, list(synth.config1(seed=82, L=600).triplets)),
             (synth.protein_scoring(83), list(synth.config3(seed=83, L=420).triplets))]
    for sc, trips in cases:
        plan = _semi_plan(sc, tile, flags)
        try:
            bt = B.trioseq_batch_create(plan, [strs(trips[0], sc)])
            try:
                info = B.trioseq_batch_info(bt)
                assert info["kernel"].startswith("wavefront_vl_kernel"), info
            finally:
                B.trioseq_batch_destroy(bt)
            got = B.trioseq_align_batch(plan, [strs(t, sc) for t in trips])
            want = [oracle.align_type(*t, sc.sub, sc.gap, kind) for t in trips]
            assert got.tolist() == want
            for t, w in list(zip(trips, want))[:3]:  # alone as well as in the batch
                assert int(B.trioseq_align_batch(plan, [strs(t, sc)])[0]) == w
        finally:
            B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", ["8x16", "8x8v"])
@pytest.mark.parametrize("flags", [B.SEMIGLOBAL, B.LOCAL], ids=["semiglobal", "local"])
def test_vl_variant_types_full_size_equal_int32(tile, flags):
    """The n=4000 protein triplet, semi-global and local: the two-per-register kernel equals the
    int32 kernel (itself exact against the oracle on every smaller case)."""
    w = synth.config3()
    s = [strs(t, w.scoring) for t in w.triplets]
    ref, vl = _semi_plan(w.scoring, "8x8", flags), _semi_plan(w.scoring, tile, flags)
    try:
        assert B.trioseq_align_batch(vl, s).tolist() == B.trioseq_align_batch(ref, s).tolist()
    finally:
        B.trioseq_plan_destroy(vl)
        B.trioseq_plan_destroy(ref)
