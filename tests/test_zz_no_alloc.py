"""The allocation-free entry point (trioseq_align_noalloc), through the C ABI.

It serves callers that may not allocate device memory when they align (their device memory is
already reserved by another allocator, or their host forbids cudaMalloc in callbacks): its
workspace is a fixed array in the library. Its score must equal the oracle's and the regular
entry point's (trioseq_align_batch, score only) exactly, on consecutive calls that reuse the same
array.
This file is collected last so that a run stopping at the first failure has run every other
test first.
"""
import numpy as np
import pytest

from paper_2605_28400_gb300 import binding as B
from paper_2605_28400_gb300 import synth

pytestmark = pytest.mark.gpu


def _device_bytes(torch, s: str):
    if not s:
        return torch.empty(0, dtype=torch.uint8, device="cuda")
    return torch.tensor(np.frombuffer(s.encode(), dtype=np.uint8).copy(), device="cuda")


def _noalloc(torch, sc, strs):
    d = [_device_bytes(torch, s) for s in strs]
    out = torch.full((1,), -123456789, dtype=torch.int32, device="cuda")
    st = B.trioseq_align_noalloc(sc.alphabet, sc.sub, sc.gap,
                                 d[0].data_ptr() if len(strs[0]) else 0, len(strs[0]),
                                 d[1].data_ptr() if len(strs[1]) else 0, len(strs[1]),
                                 d[2].data_ptr() if len(strs[2]) else 0, len(strs[2]),
                                 out.data_ptr(), torch.cuda.current_stream())
    return st, int(out.item())


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    cases = [(synth.dna_scoring(), synth.config1(seed=501, L=420).triplets[0]),
             (synth.dna_scoring(), synth.config2(seed=502, n=1, lo=60, hi=60).triplets[0]),
             (synth.protein_scoring(503), synth.config3(seed=503, L=250).triplets[0])]
    for sc, trip in cases:
        strs = [synth.to_str(s, sc.alphabet) for s in trip]
        plan = B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
        try:
            want = int(B.trioseq_align_batch(plan, [strs], B.SCORE_ONLY)[0])
        finally:
            B.trioseq_plan_destroy(plan)
        for _ in range(2):  # two calls in a row on the shared array
            st, got = _noalloc(torch, sc, strs)
            assert st == B.OK, B.trioseq_strerror(st)
            assert got == want


def test_noalloc_edge_cases_and_limits():
    torch = pytest.importorskip("torch")
    torch.cuda.set_device(0)
    sc = synth.dna_scoring()
    st, got = _noalloc(torch, sc, ["ACGT", "", "ACG"])
    plan = B.trioseq_plan(sc.alphabet, sc.sub, sc.gap)
    try:
        want = int(B.trioseq_align_batch(plan, [["ACGT", "", "ACG"]])[0])
    finally:
        B.trioseq_plan_destroy(plan)
    assert st == B.OK and got == want
    st, _ = _noalloc(torch, sc, ["ACGX", "A", "C"])
    assert st == B.EINVAL
    big = "A" * 4000
    st, _ = _noalloc(torch, sc, [big, big, big])  # workspace far beyond the fixed array
    assert st == B.ESCRATCH
    st, got = _noalloc(torch, sc, ["AC", "AC", "AC"])  # usable again after the rejections
    assert st == B.OK and got == 3 * 2 * 2


def test_noalloc_equals_the_oracle():
    """Scores straight against oracle.align (Eq. 1, Sec. II): every shape up to 3^3 with random
    DNA residues, ragged shapes that span several column tasks, and a protein case."""
    torch = pytest.importorskip("torch")
    import itertools

    import oracle
    torch.cuda.set_device(0)
    rng = np.random.default_rng(511)
    dna, prot = synth.dna_scoring(), synth.protein_scoring(512)
    cases = [(dna, s) for s in itertools.product(range(4), repeat=3)]
    cases += [(dna, s) for s in ((37, 70, 55), (90, 12, 64), (0, 60, 61), (130, 97, 41))]
    cases += [(prot, (80, 75, 90))]
    bad = []
    for sc, shape in cases:
        trip = [rng.integers(0, len(sc.alphabet), n).astype(np.uint8) for n in shape]
        st, got = _noalloc(torch, sc, [synth.to_str(s, sc.alphabet) for s in trip])
        want = oracle.align(*trip, sc.sub, sc.gap)
        if st != B.OK or got != want:
            bad.append((shape, st, got, want))
    assert not bad, bad[:5]
