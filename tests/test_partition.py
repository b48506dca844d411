"""trioseq_partition, the Sec. V-D work partitioning over ranks (host only, no GPU).

Checked: blocked and interleaved against their definitions, plus contiguity and balance in count;
dynamic by replaying its rule (each triplet goes to a least-loaded rank, lowest first), by Graham's
bound for greedy list scheduling (max load <= mean load + the largest triplet), and by the
paper's two synthetic dataset shapes, each ideal for one static scheme and poor for the other,
on which dynamic stays balanced; largest first by replaying it on the sorted order and by
Graham's LPT bound (4/3 - 1/(3N) times the optimum, found by brute force on small sets); argument
errors and the 64-bit overflow check.
"""
import itertools

import numpy as np
import pytest

from paper_2605_28400_gb300 import binding as B


def cells(lens):
    lens = np.asarray(lens, dtype=np.int64).reshape(-1, 3)
    return lens[:, 0] * lens[:, 1] * lens[:, 2]


def rand_lens(seed, n, hi=300):
    return np.random.default_rng(seed).integers(0, hi, size=(n, 3))


@pytest.mark.parametrize("n,N", [(0, 1), (1, 1), (5, 8), (10, 3), (4096, 8), (999, 7)])
def test_blocked_and_interleaved_definitions(n, N):
    lens = rand_lens(n + N, n)
    c = cells(lens)
    blk, lb = B.trioseq_partition(lens, N, B.PART_BLOCKED)
    itl, li = B.trioseq_partition(lens, N, B.PART_INTERLEAVED)
    t = np.arange(n)
    assert itl.tolist() == (t % N).tolist()
    # blocked: non-decreasing ranks, chunk r = [floor(r n/N), floor((r+1) n/N))
    assert (np.diff(blk) >= 0).all()
    for r in range(N):
        assert np.flatnonzero(blk == r).tolist() == list(range(r * n // N, (r + 1) * n // N))
    sizes = np.bincount(blk, minlength=N)
    assert sizes.max() - sizes.min() <= 1 if n else sizes.sum() == 0
    for ranks, load in ((blk, lb), (itl, li)):
        assert load.tolist() == [int(c[ranks == r].sum()) for r in range(N)]


def replay_dynamic(c, N):
    load = [0] * N
    out = []
    for x in c:
        r = min(range(N), key=lambda q: (load[q], q))
        out.append(r)
        load[r] += int(x)
    return out, load


@pytest.mark.parametrize("seed,n,N", [(1, 50, 2), (2, 4096, 8), (3, 300, 7), (4, 3, 8)])
def test_dynamic_is_least_cumulative_cells_first(seed, n, N):
    lens = rand_lens(seed, n)
    lens[::17] = 0  # empty triplets: zero work, they go to the least-loaded, lowest rank
    c = cells(lens)
    got, load = B.trioseq_partition(lens, N, B.PART_DYNAMIC)
    want, want_load = replay_dynamic(c, N)
    assert got.tolist() == want
    assert load.tolist() == want_load
    # Graham's bound for greedy list scheduling
    assert load.max() <= c.sum() / N + (c.max() if n else 0)


def test_dynamic_default_scheme():
    lens = rand_lens(5, 64)
    assert B.trioseq_partition(lens, 4)[0].tolist() == \
        B.trioseq_partition(lens, 4, B.PART_DYNAMIC)[0].tolist()


def imbalance(load):
    return float(load.max()) / float(load.mean())


def test_dataset_shapes_of_sec_v_d():
    """Sec. V-D's first dataset suits blocked partitioning and its second interleaved; the wrong
    static scheme loses badly on each, while dynamic partitioning stays near balance on both.
    Periodic lengths (period N) are balanced by blocked and piled onto few ranks by interleaved;
    lengths rising in runs of N (each run one length) are the reverse."""
    N, per = 8, 64
    rng = np.random.default_rng(9)
    L = rng.integers(60, 400, size=N)
    periodic = np.repeat(L[np.arange(N * per) % N][:, None], 3, axis=1)
    runs = np.repeat(np.repeat(np.sort(rng.integers(60, 400, size=per)), N)[:, None], 3, axis=1)
    lp = {s: B.trioseq_partition(periodic, N, s)[1] for s in (0, 1, 2)}
    lr = {s: B.trioseq_partition(runs, N, s)[1] for s in (0, 1, 2)}
    assert imbalance(lp[B.PART_BLOCKED]) < 1.001 and imbalance(lp[B.PART_INTERLEAVED]) > 1.5
    assert imbalance(lr[B.PART_INTERLEAVED]) < 1.001 and imbalance(lr[B.PART_BLOCKED]) > 1.5
    assert imbalance(lp[B.PART_DYNAMIC]) < 1.05 and imbalance(lr[B.PART_DYNAMIC]) < 1.05


def test_errors():
    lens = rand_lens(6, 4)
    for nranks, scheme in ((0, 0), (-1, 2), (2, 4), (2, -1)):
        with pytest.raises(B.TrioseqError) as e:
            B.trioseq_partition(lens, nranks, scheme)
        assert e.value.status == B.EINVAL
    big = np.full((2, 3), 0xFFFFFFFF, dtype=np.uint32)  # (2^32 - 1)^3 cells: above 2^64
    with pytest.raises(B.TrioseqError) as e:
        B.trioseq_partition(big, 2)
    assert e.value.status == B.EOVERFLOW
    # 2^21 cubed = 2^63 per triplet: one fits, and two sum to exactly 2^64, which does not
    ok = np.full((1, 3), 1 << 21, dtype=np.uint32)
    assert B.trioseq_partition(ok, 2)[1].tolist() == [1 << 63, 0]
    with pytest.raises(B.TrioseqError) as e:
        B.trioseq_partition(np.vstack([ok, ok]), 2)
    assert e.value.status == B.EOVERFLOW


@pytest.mark.parametrize("seed,n,N", [(11, 40, 3), (12, 4096, 8), (13, 9, 4)])
def test_largest_first_is_dynamic_on_decreasing_cells(seed, n, N):
    lens = rand_lens(seed, n)
    c = cells(lens)
    order = sorted(range(n), key=lambda t: -c[t])  # stable: ties keep dataset order
    got, load = B.trioseq_partition(lens, N, B.PART_LARGEST_FIRST)
    ranks, want_load = replay_dynamic(c[order], N)
    want = [0] * n
    for t, r in zip(order, ranks):
        want[t] = r
    assert got.tolist() == want and load.tolist() == want_load


def test_largest_first_within_graham_lpt_bound_of_optimum():
    rng = np.random.default_rng(14)
    for trial in range(40):
        n, N = int(rng.integers(1, 9)), int(rng.integers(2, 4))
        lens = rng.integers(1, 12, size=(n, 3))
        c = cells(lens)
        opt = min(max(sum(int(c[t]) for t in range(n) if a[t] == r) for r in range(N))
                  for a in itertools.product(range(N), repeat=n))
        got = int(B.trioseq_partition(lens, N, B.PART_LARGEST_FIRST)[1].max())
        assert opt <= got <= (4 / 3 - 1 / (3 * N)) * opt + 1e-9


def test_heavy_tailed_set_balances_better_largest_first():
    """Lengths lognormal(ln 300, 0.8) clipped to [50, 2000] (the serving mix): in dataset order a
    few very large triplets late in the set unbalance the dynamic scheme; largest first does not."""
    rng = np.random.default_rng(2024)
    lens = np.clip(np.exp(rng.normal(np.log(300), 0.8, size=(4096, 3))), 50, 2000).astype(int)
    for N in (8, 64):
        dyn = B.trioseq_partition(lens, N, B.PART_DYNAMIC)[1]
        lpt = B.trioseq_partition(lens, N, B.PART_LARGEST_FIRST)[1]
        assert lpt.max() <= dyn.max()
        assert imbalance(lpt) < 1.02
