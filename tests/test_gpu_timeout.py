"""Bounded device waits: a wait that sees no progress gives up, the call reports ETIMEOUT, and the
CUDA context stays usable. The test makes a wait run out without any GPU fault: with
TRIOSEQ_TEST_WAIT_UNSET the first-wave column tasks wait on a progress word that nothing writes,
and TRIOSEQ_WAIT_MS shortens the limit to 20 ms."""
import os

import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu

DNA = synth.dna_scoring()


def _plan(env):
    saved = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return B.trioseq_plan(DNA.alphabet, DNA.sub, DNA.gap)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def test_expired_wait_reports_etimeout_and_context_stays_usable():
    rng = np.random.default_rng(41)
    trips = [tuple(rng.integers(0, 4, size=n).astype(np.uint8) for n in (300, 280, 310)),
             tuple(rng.integers(0, 4, size=n).astype(np.uint8) for n in (90, 120, 60))]
    strs = [[synth.to_str(s, DNA.alphabet) for s in t] for t in trips]
    stalled = _plan({"TRIOSEQ_TEST_WAIT_UNSET": 1, "TRIOSEQ_WAIT_MS": 20})
    try:
        with pytest.raises(B.TrioseqError) as exc:
            B.trioseq_align_batch(stalled, strs)
        assert exc.value.status == B.ETIMEOUT
    finally:
        B.trioseq_plan_destroy(stalled)
    plan = _plan({})
    try:  # the same device and process keep working, with exact results
        got = B.trioseq_align_batch(plan, strs)
        assert got.tolist() == oracle.align_many(trips, DNA.sub, DNA.gap).tolist()
    finally:
        B.trioseq_plan_destroy(plan)
