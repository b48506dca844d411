"""Host-side fault injection and limits, through the C ABI: integer-range overflow, an injected
device allocation failure, and a full server queue. Each failure must come back as its status
code, and the library must keep working afterwards. No GPU fault is made: the overflow checks
run on the host before any launch, the allocation failure is injected in the allocation wrapper
(TRIOSEQ_TEST_FAIL_ALLOC), and the queue limit comes from TRIOSEQ_SERVER_MAX_PENDING."""
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()


def _with_env(env, fn):
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return fn()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _status(fn):
    with pytest.raises(B.TrioseqError) as exc:
        fn()
    return exc.value.status


def test_integer_range_overflow_is_rejected_before_launch():
    plan = B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap)
    semi = B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap, B.SEMIGLOBAL)
    try:
        # a sequence longer than 2^24 residues
        assert _status(lambda: B.trioseq_align_batch(
            plan, [("A" * ((1 << 24) + 1), "A", "A")])) == B.EOVERFLOW
        # traceback keys need max|sigma''| * (a+b+c) below 2^26: 6 * 3 * 3.8M is not
        long = "ACGT" * 950_000
        assert _status(lambda: B.trioseq_align_batch(plan, [(long, long, long)])) == B.EOVERFLOW
        # semi-global / local traceback: the best cell's index needs (a+1)(b+1)(c+1) < 2^37
        s = "ACGT" * 1300
        assert _status(lambda: B.trioseq_align_batch(semi, [(s, s, s)], B.WITH_TRACEBACK)) \
            == B.EOVERFLOW
        # the plans still align, exactly
        t = tuple(np.array([DNA.alphabet.index(ch) for ch in x], dtype=np.uint8)
                  for x in ("ACGTTGCA", "ACGTGCA", "AGTTGCA"))
        got = B.trioseq_align_batch(plan, [[synth.to_str(x, DNA.alphabet) for x in t]])
        assert int(got[0]) == oracle.align(*t, DNA.sub, DNA.gap)
    finally:
        B.trioseq_plan_destroy(semi)
        B.trioseq_plan_destroy(plan)


def test_injected_allocation_failure_reports_enomem():
    rng = np.random.default_rng(43)
    trips = [tuple(rng.integers(0, 4, size=n).astype(np.uint8) for n in (90, 70, 80))]
    strs = [[synth.to_str(s, DNA.alphabet) for s in t] for t in trips]
    # the first device allocation after this plan's creation fails: the batch's workspace
    failing = _with_env({"TRIOSEQ_TEST_FAIL_ALLOC": 1},
                        lambda: B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap))
    try:
        assert _status(lambda: B.trioseq_align_batch(failing, strs)) == B.ENOMEM
        # the next allocation succeeds: the same plan recovers
        got = B.trioseq_align_batch(failing, strs)
        assert got.tolist() == oracle.align_many(trips, DNA.sub, DNA.gap).tolist()
    finally:
        B.trioseq_plan_destroy(failing)


def test_full_server_queue_reports_eagain():
    plan = B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap)
    srv = _with_env({"TRIOSEQ_SERVER_MAX_PENDING": 0}, lambda: B.trioseq_server_create([plan]))
    try:
        st, _ = B.trioseq_submit(srv, ["ACGT" * 10, "ACGA" * 10, "AGGT" * 10], 0)
        assert st == B.EAGAIN
    finally:
        B.trioseq_server_destroy(srv)
        B.trioseq_plan_destroy(plan)
