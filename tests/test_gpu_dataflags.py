"""Boundary records as their own readiness flags (traceback launches).

One-triplet traceback launches fill their boundary records with a sentinel before the launch and
let a consumer wait on the record slots it stages instead of on its producers' progress words.
Scores and alignments must equal the oracle's with the scheme on (the default for one triplet),
forced on for multi-triplet batches, and forced off; every traceback tile is covered. A wait on
records that never come runs out (bounded, no fault) and the call reports ETIMEOUT.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()


def _plan(sc, **env):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _text(rows, sc):
    return tuple("".join("-" if v == 255 else sc.alphabet[v] for v in r) for r in rows)


@pytest.mark.parametrize("tile", ["8x4", "4x8", "8x8", "4x4"])
@pytest.mark.parametrize("flags", [None, 0], ids=["default", "off"])
def test_one_triplet_traceback_exact(tile, flags):
    cases = [(DNA, synth.config1(seed=91, L=420).triplets[0]),
             (synth.protein_scoring(92), synth.config3(seed=92, L=230).triplets[0])]
    for sc, t in cases:
        env = {"TRIOSEQ_TB_TILE": tile}
        if flags is not None:
            env["TRIOSEQ_DATA_FLAGS"] = flags
        plan = _plan(sc, **env)
        try:
            got = B.trioseq_align_batch(plan, [[synth.to_str(s, sc.alphabet) for s in t]],
                                        B.WITH_TRACEBACK)
            score, rows = oracle.align(*t, sc.sub, sc.gap, traceback=True)
            assert int(got[0]) == score
            assert B.trioseq_traceback(plan, 0) == _text(rows, sc)
        finally:
            B.trioseq_plan_destroy(plan)


def test_forced_on_for_a_batch_and_resident_reruns():
    w = synth.config2(seed=93, n=40, lo=20, hi=160)
    strs = [[synth.to_str(s, w.scoring.alphabet) for s in t] for t in w.triplets]
    plan = _plan(w.scoring, TRIOSEQ_DATA_FLAGS=1)
    try:
        bt = B.trioseq_batch_create(plan, strs, B.WITH_TRACEBACK)
        try:
            for _ in range(2):  # the sentinel fill is part of every run (graph replay included)
                B.trioseq_batch_run(bt)
                got = B.trioseq_batch_scores(bt, len(strs))
                for i in (0, 7, 39):
                    score, rows = oracle.align(*w.triplets[i], w.scoring.sub, w.scoring.gap,
                                               traceback=True)
                    assert int(got[i]) == score
                    assert B.trioseq_batch_alignment(bt, i) == _text(rows, w.scoring)
            assert got.tolist() == oracle.align_many(w.triplets, w.scoring.sub,
                                                     w.scoring.gap).tolist()
        finally:
            B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)


def test_records_that_never_come_time_out():
    """First-wave tasks wait on a progress word nothing writes (TRIOSEQ_TEST_WAIT_UNSET) and give
    up. The triplet has more tasks than resident warps (4x4 tile, ancestor 1200), so later tasks
    start without that wait and then wait on records their given-up producers never write: they
    give up after the 20 ms limit too, and the call reports ETIMEOUT. The same process then
    aligns exactly (equal to the flag-polling path, which the oracle pins elsewhere)."""
    t = synth.config1(seed=94, L=1200).triplets[0]
    s = [[synth.to_str(x, DNA.alphabet) for x in t]]
    plan = _plan(DNA, TRIOSEQ_TEST_WAIT_UNSET=1, TRIOSEQ_WAIT_MS=20, TRIOSEQ_TB_TILE="4x4")
    try:
        bt = B.trioseq_batch_create(plan, s, B.WITH_TRACEBACK)
        try:
            assert B.trioseq_batch_info(bt)["tasks"] > 152 * 4 * 4  # beyond the first wave
        finally:
            B.trioseq_batch_destroy(bt)
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_align_batch(plan, s, B.WITH_TRACEBACK)
        assert e.value.status == B.ETIMEOUT
    finally:
        B.trioseq_plan_destroy(plan)
    on, off = _plan(DNA), _plan(DNA, TRIOSEQ_DATA_FLAGS=0)
    try:
        got = B.trioseq_align_batch(on, s, B.WITH_TRACEBACK)
        want = B.trioseq_align_batch(off, s, B.WITH_TRACEBACK)
        assert got.tolist() == want.tolist()
        assert B.trioseq_traceback(on, 0) == B.trioseq_traceback(off, 0)
    finally:
        B.trioseq_plan_destroy(on)
        B.trioseq_plan_destroy(off)
