"""Serving through submit/poll: continuous batching must not change any result.

A mixed stream (DNA and protein scoring, score-only and traceback requests, uneven lengths) is
submitted while earlier requests are still on the GPU. Every result is compared with the same
request aligned alone through trioseq_align_batch (tolerance 0: scores and rows identical), and
a sample with the CPU oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu


def _poll_all(srv, tickets, cap, timeout_s=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for tk in tickets:
            if tk in out:
                continue
            st, score, rows = B.trioseq_poll(srv, tk, cap)
            if st == B.OK:
                out[tk] = (score, rows)
        assert time.time() - t0 < timeout_s, "serving did not finish in time"
        time.sleep(0.0005)
    return out


def test_mixed_stream_equals_alone():
    dna, prot = synth.dna_scoring(), synth.protein_scoring(1004)
    plans = [B.trioseq_plan(dna.alphabet, dna.sub, dna.gap),
             B.trioseq_plan(prot.alphabet, prot.sub, prot.gap)]
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(48):
        protein = bool(i % 3 == 2)
        sc = prot if protein else dna
        L = int(rng.integers(10, 220))
        trip = synth.related_triplet(99, i, L, sc, 0.1, 0.03, 2.0)
        reqs.append((1 if protein else 0, bool(i % 5 == 0), trip, sc))
    srv = B.trioseq_server_create(plans)
    try:
        tickets = []
        for pid, tb, trip, sc in reqs:
            st, tk = B.trioseq_submit(srv, [synth.to_str(s, sc.alphabet) for s in trip], pid,
                                      B.WITH_TRACEBACK if tb else B.SCORE_ONLY)
            assert st == B.OK
            tickets.append(tk)
        cap = 3 * 300
        got = _poll_all(srv, tickets, cap)
        # a consumed ticket is unknown afterwards
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_poll(srv, tickets[0], cap)
        assert e.value.status == B.EINVAL
    finally:
        B.trioseq_server_destroy(srv)
    try:
        for (pid, tb, trip, sc), tk in zip(reqs, tickets):
            strs = [synth.to_str(s, sc.alphabet) for s in trip]
            alone = B.trioseq_align_batch(plans[pid], [strs],
                                          B.WITH_TRACEBACK if tb else B.SCORE_ONLY)
            score, rows = got[tk]
            assert score == int(alone[0])
            if tb:
                assert rows == B.trioseq_traceback(plans[pid], 0)
        for (pid, tb, trip, sc), tk in list(zip(reqs, tickets))[:6]:
            assert got[tk][0] == oracle.align(*trip, sc.sub, sc.gap)
    finally:
        for p in plans:
            B.trioseq_plan_destroy(p)


def test_server_rejects_bad_requests():
    dna = synth.dna_scoring()
    plan = B.trioseq_plan(dna.alphabet, dna.sub, dna.gap)
    srv = B.trioseq_server_create([plan])
    try:
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_submit(srv, ["ACGN", "A", "C"], 0)
        assert e.value.status == B.EINVAL
        with pytest.raises(B.TrioseqError):
            B.trioseq_submit(srv, ["ACG", "A", "C"], 5)  # unknown plan
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_poll(srv, 123456789, 0)
        assert e.value.status == B.EINVAL
        st, tk = B.trioseq_submit(srv, ["ACGT" * 30, "ACGA" * 30, "AGGT" * 30], 0)
        assert st == B.OK
        got = _poll_all(srv, [tk], 0)
        plan_alone = B.trioseq_align_batch(plan, [["ACGT" * 30, "ACGA" * 30, "AGGT" * 30]])
        assert got[tk][0] == int(plan_alone[0])
    finally:
        B.trioseq_server_destroy(srv)
        B.trioseq_plan_destroy(plan)


def test_variant_plans_served_with_traceback():
    # a server over a local-type DNA plan and a semi-global protein plan, traceback requests
    # included: every result equals the oracle's alignment of its type
    dna, prot = synth.dna_scoring(), synth.protein_scoring(1005)
    plans = [B.trioseq_plan(dna.alphabet, dna.sub, dna.gap, B.LOCAL),
             B.trioseq_plan(prot.alphabet, prot.sub, prot.gap, B.SEMIGLOBAL)]
    kinds = [oracle.LOCAL, oracle.SEMIGLOBAL]
    rng = np.random.default_rng(8)
    reqs = []
    for i in range(24):
        pid = i % 2
        sc = prot if pid else dna
        trip = tuple(rng.integers(0, sc.sub.shape[0], size=int(rng.integers(5, 90))).astype(
            np.uint8) for _ in range(3))
        reqs.append((pid, bool(i % 3 == 0), trip, sc))
    srv = B.trioseq_server_create(plans)
    try:
        tickets = []
        for pid, tb, trip, sc in reqs:
            st, tk = B.trioseq_submit(srv, [synth.to_str(s, sc.alphabet) for s in trip], pid,
                                      B.WITH_TRACEBACK if tb else B.SCORE_ONLY)
            assert st == B.OK
            tickets.append(tk)
        got = _poll_all(srv, tickets, 3 * 100)
    finally:
        B.trioseq_server_destroy(srv)
        for p in plans:
            B.trioseq_plan_destroy(p)
    for (pid, tb, trip, sc), tk in zip(reqs, tickets):
        score, rows, _, _ = oracle.align_type_tb(*trip, sc.sub, sc.gap, kinds[pid])
        got_score, got_rows = got[tk]
        assert got_score == score
        if tb:  # an empty alignment comes back as no rows
            assert (got_rows or ("", "", "")) == tuple(
                "".join("-" if v == 255 else sc.alphabet[v] for v in r) for r in rows)


def test_request_beyond_a_launch_share_waits_for_room_and_is_exact():
    """Admission shares one device-memory budget among the launches in flight. With a 64 MiB
    budget, a quarter (one launch's share of small requests) is 16 MiB. A 600-residue triplet
    needs about 46 MiB of workspace: it must wait for room among small requests and complete
    exactly (oracle). An 800-residue triplet needs about 108 MiB, more than the whole budget:
    it completes with ENOMEM while everything around it still completes exactly."""
    dna = synth.dna_scoring()
    plan = B.trioseq_plan(dna.alphabet, dna.sub, dna.gap)
    small = [synth.related_triplet(77, i, 90 + 7 * i, dna, 0.05, 0.02, 2.0) for i in range(12)]
    mid = synth.related_triplet(78, 0, 600, dna, 0.05, 0.02, 2.0)
    huge = synth.related_triplet(79, 0, 800, dna, 0.05, 0.02, 2.0)
    order = small[:6] + [mid] + small[6:9] + [huge] + small[9:]
    srv = B.trioseq_server_create([plan], hbm_budget=64 << 20)
    try:
        tickets = []
        for i, trip in enumerate(order):
            mode = B.WITH_TRACEBACK if i % 4 == 1 else B.SCORE_ONLY
            st, tk = B.trioseq_submit(srv, [synth.to_str(s, dna.alphabet) for s in trip], 0, mode)
            assert st == B.OK
            tickets.append((tk, mode))
        huge_tk = tickets[next(i for i, t in enumerate(order) if t is huge)][0]
        rest = [tk for tk, _ in tickets if tk != huge_tk]
        got = _poll_all(srv, rest, 3 * 700)
        t0 = time.time()
        while True:
            try:
                st, _, _ = B.trioseq_poll(srv, huge_tk, 0)
            except B.TrioseqError as e:
                assert e.status == B.ENOMEM
                break
            assert st == B.EAGAIN and time.time() - t0 < 60
            time.sleep(0.001)
    finally:
        B.trioseq_server_destroy(srv)
    try:
        for (tk, mode), trip in zip(tickets, order):
            if tk == huge_tk:
                continue
            score, rows = got[tk]
            if mode == B.WITH_TRACEBACK:
                want, wrows = oracle.align(*trip, dna.sub, dna.gap, traceback=True)
                assert rows == tuple("".join("-" if v == 255 else dna.alphabet[v] for v in r)
                                     for r in wrows)
            else:
                want = oracle.align(*trip, dna.sub, dna.gap)
            assert score == want
    finally:
        B.trioseq_plan_destroy(plan)
