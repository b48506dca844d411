"""GPU parity of the sharded batch path: a batch split over ranks by trioseq_partition, each share
aligned by its own plan in its own launch (as each rank of a multi-GPU run does), gives, put back
in dataset order, exactly the oracle's scores for the whole batch. The ranks run one after another
on the one GPU; no rank waits on another."""
import numpy as np
import pytest

import oracle
from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("world,scheme", [(2, B.PART_LARGEST_FIRST), (3, B.PART_DYNAMIC),
                                          (4, B.PART_BLOCKED), (5, B.PART_INTERLEAVED)])
def test_shards_put_back_equal_the_oracle(world, scheme):
    w = synth.config2(seed=31, n=48, lo=10, hi=90)
    sc = w.scoring
    strs = [[synth.to_str(s, sc.alphabet) for s in t] for t in w.triplets]
    lens = [[len(s) for s in t] for t in w.triplets]
    rank_of, cells = B.trioseq_partition(lens, world, scheme)
    got = np.zeros(len(strs), dtype=np.int64)
    for r in range(world):
        idx = np.flatnonzero(rank_of == r)
        assert int(cells[r]) == sum(lens[t][0] * lens[t][1] * lens[t][2] for t in idx)
        if idx.size == 0:
            continue
        plan = B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
        try:
            got[idx] = B.trioseq_align_batch(plan, [strs[t] for t in idx])
        finally:
            B.trioseq_plan_destroy(plan)
    want = oracle.align_many(w.triplets, sc.sub, sc.gap)
    assert got.tolist() == want.tolist()
