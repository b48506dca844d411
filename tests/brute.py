"""Brute-force 3-way alignment by enumeration (pins the oracle; tiny inputs only).

Independent of any dynamic program: it walks every monotone lattice path from (a, b, c) back to
the origin, one column per step (each column consumes one residue from a non-empty subset of the
three sequences), and scores each complete alignment column by column with the sum-of-pairs
definition of Sec. II (sigma(residue, gap) = alpha, sigma(gap, gap) = 0).

Moves are tried in Eq. 1's listing order at every step, walking from the END of the alignment.
The depth-first search therefore meets the alignments in lexicographic order of their reversed
move sequences, and the first alignment reaching the final maximum is the one a traceback with
the "first maximal move in Eq. 1's order wins" tie-break emits.
"""
from __future__ import annotations

GAP = 255
MOVES = ((1, 1, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 0, 0), (0, 1, 0), (0, 0, 1))


def _sigma(x, y, sub, gap):
    if x is None and y is None:
        return 0
    if x is None or y is None:
        return gap
    return int(sub[x][y])


def column_score(col, sub, gap):
    x, y, z = col
    return _sigma(x, y, sub, gap) + _sigma(x, z, sub, gap) + _sigma(y, z, sub, gap)


def count_alignments(a, b, c):
    """Number of distinct 3-way alignments (monotone lattice paths with the 7 moves)."""
    memo = {}

    def f(i, j, k):
        if i == 0 and j == 0 and k == 0:
            return 1
        if (i, j, k) in memo:
            return memo[(i, j, k)]
        t = 0
        for di, dj, dk in MOVES:
            if i >= di and j >= dj and k >= dk:
                t += f(i - di, j - dj, k - dk)
        memo[(i, j, k)] = t
        return t

    return f(a, b, c)


def brute_force(s0, s1, s2, sub, gap):
    """Return (best score, tie-break-first optimal alignment as 3 lists with GAP for gaps)."""
    s = [list(map(int, s0)), list(map(int, s1)), list(map(int, s2))]
    best = [None, None]
    cols = []

    def rec(i, j, k, acc):
        if i == 0 and j == 0 and k == 0:
            if best[0] is None or acc > best[0]:
                best[0] = acc
                best[1] = list(reversed(cols))
            return
        for di, dj, dk in MOVES:
            if i < di or j < dj or k < dk:
                continue
            col = (s[0][i - 1] if di else None, s[1][j - 1] if dj else None,
                   s[2][k - 1] if dk else None)
            cols.append(col)
            rec(i - di, j - dj, k - dk, acc + column_score(col, sub, gap))
            cols.pop()

    rec(len(s[0]), len(s[1]), len(s[2]), 0)
    rows = [[GAP if col[q] is None else col[q] for col in best[1]] for q in range(3)]
    return best[0], rows


def brute_best_ending_at(s0, s1, s2, sub, gap, end, kind):
    """Best score of an alignment path that ends at cell `end` and starts where the alignment type
    allows: any cell s <= end for local (the empty path scores 0), an axis cell (two zero
    indices) for semi-global. Enumerates every start and every path (tiny inputs only)."""
    i1, j1, k1 = end
    best = 0 if kind == 2 else None
    for i0 in range(i1 + 1):
        for j0 in range(j1 + 1):
            for k0 in range(k1 + 1):
                if kind == 1 and (i0 == 0) + (j0 == 0) + (k0 == 0) < 2:
                    continue
                v, _ = brute_force(s0[i0:i1], s1[j0:j1], s2[k0:k1], sub, gap)
                best = v if best is None else max(best, v)
    return best


def brute_walk(s0, s1, s2, sub, gap, end, kind, target):
    """First path (in the order: moves by Eq. 1's listing, then stopping) that walks back from
    `end` to a start with total score `target`. Starts: axis cells always (they are initialised);
    for local also any cell (v = 0, listed after the moves). Returns (rows, begin)."""
    s = [list(map(int, s0)), list(map(int, s1)), list(map(int, s2))]
    cols = []
    found = [None]

    def rec(i, j, k, acc):
        axis = (i == 0) + (j == 0) + (k == 0) >= 2
        if not axis:
            for di, dj, dk in MOVES:
                if i < di or j < dj or k < dk:
                    continue
                col = (s[0][i - 1] if di else None, s[1][j - 1] if dj else None,
                       s[2][k - 1] if dk else None)
                cols.append(col)
                if rec(i - di, j - dj, k - dk, acc + column_score(col, sub, gap)):
                    return True
                cols.pop()
        if (axis or kind == 2) and acc == target:
            rows = [[GAP if c[q] is None else c[q] for c in reversed(cols)] for q in range(3)]
            found[0] = (rows, (i, j, k))
            return True
        return False

    rec(*end, 0)
    return found[0]
