"""Every kernel against the oracle with its boundary-record workspace poisoned.

With TRIOSEQ_TEST_POISON=1 at plan creation, each upload fills the boundary records (and slab
planes) with 0x3F3F3F3F, a value far above any score. A kernel that reads a record slot its
producer never wrote, or reads it before the producer's release, then returns a wrong score or
alignment instead of one that freshly zeroed device memory would hide. Cases: ragged multi-block
batches on every score tile (int32, two triplets per register, two cells per register), every
traceback tile, the semi-global and local types, and slab launches. Tolerance 0.
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
SHAPES = [(37, 70, 130), (129, 33, 65), (0, 100, 100), (64, 64, 0), (200, 1, 250),
          (31, 32, 63), (33, 65, 129), (17, 127, 128), (40, 135, 257), (1, 1, 1)]


def _plan(sc, flags=0, **env):
    keys = ("TRIOSEQ_TEST_POISON", "TRIOSEQ_SCORE_TILE", "TRIOSEQ_TB_TILE", "TRIOSEQ_PACKED",
            "TRIOSEQ_SLAB_SLICES")
    old = {k: os.environ.get(k) for k in keys}
    os.environ["TRIOSEQ_TEST_POISON"] = "1"
    for k, v in env.items():
        os.environ[k] = str(v)
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap, flags)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _trips(seed, sc):
    rng = np.random.default_rng(seed)
    return [tuple(rng.integers(0, len(sc.alphabet), size=n).astype(np.uint8) for n in s)
            for s in SHAPES]


def _strs(trips, sc):
    return [[synth.to_str(s, sc.alphabet) for s in t] for t in trips]


@pytest.mark.parametrize("sc", [DNA, PROT], ids=["dna", "protein"])
@pytest.mark.parametrize("env", [{"TRIOSEQ_SCORE_TILE": "8x8", "TRIOSEQ_PACKED": 0},
                                 {"TRIOSEQ_SCORE_TILE": "4x8", "TRIOSEQ_PACKED": 0},
                                 {"TRIOSEQ_SCORE_TILE": "4x4", "TRIOSEQ_PACKED": 0},
                                 {"TRIOSEQ_SCORE_TILE": "8x8"},
                                 {"TRIOSEQ_SCORE_TILE": "8x16"},
                                 {"TRIOSEQ_SCORE_TILE": "8x8v"},
                                 {"TRIOSEQ_SCORE_TILE": "8x16s"},
                                 {"TRIOSEQ_SCORE_TILE": "8x16t"}],
                         ids=["int32-8x8", "int32-4x8", "int32-4x4", "packed-8x8", "vl-8x16",
                              "vl-8x8v", "vl-8x16s", "vl-8x16t"])
def test_score_kernels_poisoned(sc, env):
    trips = _trips(61, sc)
    want = oracle.align_many(trips, sc.sub, sc.gap).tolist()
    plan = _plan(sc, **env)
    try:
        assert B.trioseq_align_batch(plan, _strs(trips, sc)).tolist() == want
        for i in (0, 6, 8):  # alone: a one-triplet batch (two cells per register for vl tiles)
            assert int(B.trioseq_align_batch(plan, _strs([trips[i]], sc))[0]) == want[i]
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", ["4x8", "8x4", "8x8", "4x4"])
def test_traceback_kernels_poisoned(tile):
    trips = _trips(62, DNA)[:6]
    plan = _plan(DNA, TRIOSEQ_TB_TILE=tile)
    try:
        got = B.trioseq_align_batch(plan, _strs(trips, DNA), B.WITH_TRACEBACK)
        for i, t in enumerate(trips):
            score, rows = oracle.align(*t, DNA.sub, DNA.gap, traceback=True)
            assert int(got[i]) == score
            want = tuple("".join("-" if v == 255 else DNA.alphabet[v] for v in r) for r in rows)
            assert (B.trioseq_traceback(plan, i) or ("", "", "")) == want
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("kind,flags", [(oracle.SEMIGLOBAL, B.SEMIGLOBAL),
                                        (oracle.LOCAL, B.LOCAL)], ids=["semiglobal", "local"])
def test_variant_types_poisoned(kind, flags):
    trips = _trips(63, PROT)
    want = [oracle.align_type(*t, PROT.sub, PROT.gap, kind) for t in trips]
    for tile in ("8x8", "8x16", "8x8v"):  # two cells per register where the type allows
        plan = _plan(PROT, flags, TRIOSEQ_SCORE_TILE=tile)
        try:
            assert B.trioseq_align_batch(plan, _strs(trips, PROT)).tolist() == want
            assert int(B.trioseq_align_batch(plan, _strs(trips[8:9], PROT))[0]) == want[8]
        finally:
            B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("mode", [B.SCORE_ONLY, B.WITH_TRACEBACK], ids=["score", "traceback"])
def test_slab_launches_poisoned(mode):
    t = synth.config1(seed=64, L=300).triplets[0]
    plan = _plan(DNA, TRIOSEQ_SLAB_SLICES=37)
    try:
        got = B.trioseq_align_batch(plan, _strs([t], DNA), mode)
        if mode == B.WITH_TRACEBACK:
            score, rows = oracle.align(*t, DNA.sub, DNA.gap, traceback=True)
            want = tuple("".join("-" if v == 255 else DNA.alphabet[v] for v in r) for r in rows)
            assert B.trioseq_traceback(plan, 0) == want
        else:
            score = oracle.align(*t, DNA.sub, DNA.gap)
        assert int(got[0]) == score
        bt = B.trioseq_batch_create(plan, _strs([t], DNA), mode)
        try:
            assert B.trioseq_batch_info(bt)["slabs"] > 1
            B.trioseq_batch_run(bt)
            assert int(B.trioseq_batch_scores(bt, 1)[0]) == score
        finally:
            B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)
