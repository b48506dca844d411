"""GPU parity at full size against stored oracle values (tests/golden, written by
tests/golden/make_goldens.py from the oracle alone).

- Config 3, the protein triplet with ancestor length 4000 (about 6.4e10 cells): its score on
  every score kernel that can take it: the two-cells-per-register tiles (8x16, 8x8v, and 8x16s
  and 8x16t with the sigma'' tile in shared memory) and the int32 8x8 kernel, through a
  device-resident batch and through trioseq_align_batch.
- Config 2, all 4,096 related DNA triplets: every score on the packed int16x2 path (the
  default), on the int32 kernel, and on the two-cells-per-register kernel.
- Config 4, the first 200 requests of the serving stream (lognormal lengths up to 2000, 30%
  protein, 20% with traceback), submitted together through trioseq_submit and harvested with
  trioseq_poll: every score, and every traceback request's alignment length and rows digest.

Tolerance 0: integer work. Each stored value is tied to its inputs by a digest, so a change in
the generators fails here instead of comparing against values of other inputs.
"""
import os
import time

import pytest

from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth
from tests.golden import goldens

pytestmark = pytest.mark.gpu


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


def _strs(trip, sc):
    return [synth.to_str(s, sc.alphabet) for s in trip]


@pytest.fixture(scope="module")
def config3():
    meta, score = goldens.load_config3()
    w = synth.config3()
    assert meta["input_sha256"] == goldens.input_digest(w.triplets), "config-3 inputs changed"
    return w, score


@pytest.mark.parametrize("tile,want_tile,want_packing", [("8x8v", (8, 8), 2), ("8x16", (8, 16), 2),
                                                         ("8x16s", (8, 16), 2),
                                                         ("8x16t", (8, 16), 2),
                                                         ("8x8", (8, 8), 1)])
def test_config3_full_size_equals_oracle(config3, tile, want_tile, want_packing):
    w, want = config3
    plan = _plan(w.scoring, TRIOSEQ_SCORE_TILE=tile)
    try:
        bt = B.trioseq_batch_create(plan, [_strs(w.triplets[0], w.scoring)])
        try:
            info = B.trioseq_batch_info(bt)
            assert info["tile"] == want_tile and info["packing"] == want_packing, info
            for _ in range(2):  # repeat runs of the same resident batch
                B.trioseq_batch_run(bt)
                assert int(B.trioseq_batch_scores(bt, 1)[0]) == want
        finally:
            B.trioseq_batch_destroy(bt)
        got = B.trioseq_align_batch(plan, [_strs(w.triplets[0], w.scoring)])
        assert int(got[0]) == want
    finally:
        B.trioseq_plan_destroy(plan)


@pytest.fixture(scope="module")
def config2():
    meta, scores = goldens.load_config2()
    w = synth.config2()
    assert meta["input_sha256"] == goldens.input_digest(w.triplets), "config-2 inputs changed"
    assert len(scores) == len(w.triplets) == 4096
    return w, scores


@pytest.mark.parametrize("env,want_packing", [({}, 2), ({"TRIOSEQ_PACKED": 0}, 1),
                                              ({"TRIOSEQ_PACKED": 0, "TRIOSEQ_SCORE_TILE": "8x16"},
                                               2)])
def test_config2_all_scores_equal_oracle(config2, env, want_packing):
    w, want = config2
    plan = _plan(w.scoring, **env)
    try:
        strs = [_strs(t, w.scoring) for t in w.triplets]
        bt = B.trioseq_batch_create(plan, strs)
        try:
            assert B.trioseq_batch_info(bt)["packing"] == want_packing
            B.trioseq_batch_run(bt)
            got = B.trioseq_batch_scores(bt, len(strs))
        finally:
            B.trioseq_batch_destroy(bt)
        bad = [i for i in range(len(want)) if int(got[i]) != int(want[i])]
        assert not bad, f"{len(bad)} scores differ, first {bad[:5]}"
    finally:
        B.trioseq_plan_destroy(plan)


def test_config4_sample_through_the_server_equals_oracle():
    meta, want = goldens.load_config4()
    dna, prot, reqs = synth.config4(n=goldens.CONFIG4_SAMPLE)
    assert meta["input_sha256"] == goldens.input_digest([r["triplet"] for r in reqs])
    plans = [B.trioseq_plan(dna.alphabet, dna.sub, dna.gap),
             B.trioseq_plan(prot.alphabet, prot.sub, prot.gap)]
    srv = B.trioseq_server_create(plans)
    try:
        tickets = []
        for r in reqs:  # all at once: later requests arrive while earlier ones are on the GPU
            sc = prot if r["protein"] else dna
            mode = B.WITH_TRACEBACK if r["traceback"] else B.SCORE_ONLY
            while True:
                st, tk = B.trioseq_submit(srv, _strs(r["triplet"], sc), int(r["protein"]), mode)
                if st != B.EAGAIN:
                    break
                time.sleep(0.001)
            assert st == B.OK, B.trioseq_strerror(st)
            tickets.append(tk)
        cap = max(sum(len(s) for s in r["triplet"]) for r in reqs)
        got = {}
        t0 = time.time()
        while len(got) < len(tickets):
            for i, tk in enumerate(tickets):
                if i in got:
                    continue
                st, score, rows = B.trioseq_poll(srv, tk, cap)
                if st == B.OK:
                    got[i] = (score, rows)
                else:
                    assert st == B.EAGAIN, B.trioseq_strerror(st)
            assert time.time() - t0 < 600, "serving did not finish in time"
            time.sleep(0.001)
    finally:
        B.trioseq_server_destroy(srv)
        for p in plans:
            B.trioseq_plan_destroy(p)
    for i, w in enumerate(want):
        assert w["id"] == reqs[i]["id"] and w["traceback"] == reqs[i]["traceback"]
        score, rows = got[i]
        assert score == w["score"], (i, score, w["score"])
        if w["traceback"]:
            assert len(rows[0]) == w["aln_len"], i
            assert goldens.rows_digest(rows) == w["rows_sha256"], i


def test_config2_affine_first_triplets_equal_oracle():
    """Affine gaps (natural gap costs) on the first 64 triplets of the config-2 batch, run in the
    whole 4,096-triplet launch: the first 64 scores equal the stored oracle values."""
    meta, want = goldens.load_config2_affine()
    w = synth.config2()
    assert meta["input_sha256"] == goldens.input_digest(w.triplets[:len(want)])
    plan = B.trioseq_plan_affine(w.scoring.alphabet, w.scoring.sub, w.scoring.gap,
                                 goldens.AFFINE_GAP_OPEN)
    try:
        got = B.trioseq_align_batch(plan, [_strs(t, w.scoring) for t in w.triplets])
    finally:
        B.trioseq_plan_destroy(plan)
    assert [int(x) for x in got[:len(want)]] == [int(x) for x in want]
