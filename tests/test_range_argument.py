"""CPU pin of the range argument behind the two-cells-per-register kernel (no GPU).

With sigma'' = sigma - 2*alpha >= 0 for every residue pair, the potential-shifted values
M'[i][j][k] = M[i][j][k] - 2*alpha*(i+j+k) of Eq. 1 are non-decreasing along each axis, and
adjacent cells differ by at most 2*max sigma''. The kernel's 16-bit relative encoding is exact
because of these two facts. Here M is computed straight from Eq. 1 (every move, out-of-cube
predecessors skipped), independently of the oracle and of the kernel, on random small cubes and
scoring schemes, including the DNA and protein schemes of the workloads.
"""
import numpy as np

from paper_2605_28400_gb300 import synth


def dp_eq1(s0, s1, s2, sub, gap):
    a, b, c = len(s0), len(s1), len(s2)
    neg = np.iinfo(np.int64).min // 4
    M = np.full((a + 1, b + 1, c + 1), neg, dtype=np.int64)
    M[0, 0, 0] = 0

    def sg(x, y):  # sigma with gaps (None) on either side
        if x is None and y is None:
            return 0
        if x is None or y is None:
            return gap
        return int(sub[x, y])

    for i in range(a + 1):
        for j in range(b + 1):
            for k in range(c + 1):
                if i == j == k == 0:
                    continue
                best = neg
                for di in (0, 1):
                    for dj in (0, 1):
                        for dk in (0, 1):
                            if not (di or dj or dk) or i < di or j < dj or k < dk:
                                continue
                            x = s0[i - 1] if di else None
                            y = s1[j - 1] if dj else None
                            z = s2[k - 1] if dk else None
                            v = M[i - di, j - dj, k - dk] + sg(x, y) + sg(x, z) + sg(y, z)
                            best = max(best, v)
                M[i, j, k] = best
    return M


def shifted(M, gap):
    a, b, c = (n - 1 for n in M.shape)
    i, j, k = np.meshgrid(np.arange(a + 1), np.arange(b + 1), np.arange(c + 1), indexing="ij")
    return M - 2 * gap * (i + j + k)


def check_bounds(s0, s1, s2, sub, gap):
    sig2 = sub.astype(np.int64) - 2 * gap
    assert (sig2 >= 0).all()
    bound = 2 * int(sig2.max())
    Mp = shifted(dp_eq1(s0, s1, s2, sub, gap), gap)
    for axis in range(3):
        d = np.diff(Mp, axis=axis)
        if d.size == 0:  # an empty sequence: no neighbours along that axis
            continue
        assert d.min() >= 0, ("not monotone", axis)
        assert d.max() <= bound, ("adjacent difference above 2 max sigma''", axis, d.max(), bound)


def test_range_argument_random_schemes():
    rng = np.random.default_rng(71)
    for trial in range(12):
        K = int(rng.integers(2, 6))
        gap = -int(rng.integers(1, 5))
        # symmetric sigma with sigma - 2*gap >= 0
        low = 2 * gap
        m = rng.integers(low, low + 12, size=(K, K))
        sub = np.triu(m) + np.triu(m, 1).T
        shape = tuple(int(x) for x in rng.integers(0, 9, size=3))
        s0, s1, s2 = (rng.integers(0, K, size=n) for n in shape)
        check_bounds(s0, s1, s2, sub, gap)


def test_range_argument_workload_schemes():
    rng = np.random.default_rng(72)
    for sc in (synth.dna_scoring(), synth.protein_scoring(1003)):
        K = len(sc.alphabet)
        sub = np.asarray(sc.sub, dtype=np.int64)
        for shape in ((7, 9, 8), (10, 4, 11), (0, 6, 9)):
            s0, s1, s2 = (rng.integers(0, K, size=n) for n in shape)
            check_bounds(s0, s1, s2, sub, sc.gap)
        # related sequences: the bound is reached along matches
        anc = rng.integers(0, K, size=9)
        check_bounds(anc, anc.copy(), np.concatenate([anc[:4], anc[5:]]), sub, sc.gap)


def test_bound_is_tight():
    """Identical sequences of one residue with sigma''(x, x) = S: the diagonal cell beside the
    axis gains exactly 2S over its neighbour along one axis."""
    sub = np.array([[6]], dtype=np.int64)
    gap = 0  # sigma'' = sigma = 6
    Mp = shifted(dp_eq1(np.zeros(3, int), np.zeros(3, int), np.zeros(3, int), sub, gap), gap)
    assert np.diff(Mp, axis=0).max() == 2 * 6
