"""GPU parity of the traceback walk on paths that stress it, against the CPU oracle, bit for bit.

The walk stages a tube of code records along the cube's diagonal and emits runs of (1,1,1) moves
32 cells at a time with warp-wide probes. These triplets make the path leave the diagonal for
long stretches (a long insertion in one sequence, a long deletion in another, indels at both
ends), run exactly along it for whole multiples of 32 cells (identical sequences), and end runs
at start cells. Every traceback tile variant and alignment type is checked, and the global type
also in slabs (linear-space traceback), where the walk resumes across slab boundaries.
"""
import functools
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()
PROT = synth.protein_scoring(1003)
TILES = ["4x4", "4x8", "8x8", "8x4"]


def _plan(sc, flags=0, tb_tile=None, slab_slices=None):
    keys = {"TRIOSEQ_TB_TILE": tb_tile, "TRIOSEQ_SLAB_SLICES": slab_slices}
    saved = {k: os.environ.get(k) for k in keys}
    for k, v in keys.items():
        if v is not None:
            os.environ[k] = str(v)
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap, flags)
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


def walk_triplets(K: int, seed: int):
    """Triplets whose optimal paths leave the diagonal for long stretches or follow it exactly."""
    rng = np.random.default_rng(seed)

    def rnd(n):
        return rng.integers(0, K, size=n).astype(np.uint8)

    anc = rnd(300)
    ins = rnd(120)
    out = [
        # long insertion in S1, long deletion in S2
        (anc, np.concatenate([anc[:140], ins, anc[140:]]), np.concatenate([anc[:60], anc[150:]])),
        # indels at both ends: extra prefix on S0, extra suffix on S2
        (np.concatenate([rnd(70), anc]), anc.copy(), np.concatenate([anc, rnd(55)])),
        # identical sequences: one run of (1,1,1) moves, whole multiples of 32 cells
        (anc[:96].copy(), anc[:96].copy(), anc[:96].copy()),
        (anc[:64].copy(), anc[:64].copy(), anc[:64].copy()),
        # one substitution at the first and at the last position
        (anc[:100].copy(), np.concatenate([[(anc[0] + 1) % K], anc[1:100]]).astype(np.uint8),
         np.concatenate([anc[:99], [(anc[99] + 1) % K]]).astype(np.uint8)),
        # unrelated sequences of very different lengths: the path hugs faces and edges
        (rnd(200), rnd(17), rnd(90)),
    ]
    return out


@functools.lru_cache(maxsize=None)
def oracle_global(name: str, seed: int):
    sc = DNA if name == "dna" else PROT
    return [oracle.align(*t, sc.sub, sc.gap, traceback=True)
            for t in walk_triplets(len(sc.alphabet), seed)]


@functools.lru_cache(maxsize=None)
def oracle_variant(kind: int, seed: int):
    return [oracle.align_type_tb(*t, DNA.sub, DNA.gap, kind) for t in walk_triplets(4, seed)]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("sc", [DNA, PROT], ids=["dna", "protein"])
def test_global_walk_stress_all_tiles(sc, tile):
    trips = walk_triplets(len(sc.alphabet), 31)
    plan = _plan(sc, tb_tile=tile)
    try:
        got = B.trioseq_align_batch(plan, [strs(t, sc) for t in trips], B.WITH_TRACEBACK)
        want = oracle_global("dna" if sc is DNA else "protein", 31)
        for i, (score, rows) in enumerate(want):
            assert int(got[i]) == score, i
            assert B.trioseq_traceback(plan, i) == rows_str(rows, sc), i
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("kinds", [(B.SEMIGLOBAL, oracle.SEMIGLOBAL), (B.LOCAL, oracle.LOCAL)],
                         ids=["semiglobal", "local"])
def test_variant_walk_stress_all_tiles(kinds, tile):
    flags, kind = kinds
    trips = walk_triplets(4, 32)
    plan = _plan(DNA, flags, tb_tile=tile)
    try:
        got = B.trioseq_align_batch(plan, [strs(t, DNA) for t in trips], B.WITH_TRACEBACK)
        for i, (score, rows, beg, end) in enumerate(oracle_variant(kind, 32)):
            assert int(got[i]) == score, i
            assert B.trioseq_traceback(plan, i) == rows_str(rows, DNA), i
            assert B.trioseq_traceback_span(plan, i) == (beg, end), i
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.mark.parametrize("slices", [37, 64])
def test_slab_walk_stress(slices):
    """Linear-space traceback: each triplet alone runs in slabs of `slices` slices; the walk
    resumes at every slab boundary, inside runs and inside long gaps alike."""
    trips = walk_triplets(4, 31)
    want = oracle_global("dna", 31)
    plan = _plan(DNA, slab_slices=slices)
    try:
        for t, (score, rows) in zip(trips[:3], want[:3]):
            got = B.trioseq_align_batch(plan, [strs(t, DNA)], B.WITH_TRACEBACK)
            assert int(got[0]) == score
            assert B.trioseq_traceback(plan, 0) == rows_str(rows, DNA)
    finally:
        B.trioseq_plan_destroy(plan)
