"""TrioSeq oracle (TEST INFRASTRUCTURE ONLY).

Python access to ``oracle.cpp``: a plain, slow CPU implementation of exact 3-way alignment
(Eq. 1 with the sum-of-pairs column score and the global initialisation of Sec. II, int64
arithmetic, first-maximal-move tie-break in Eq. 1's listing order), plus the scores of the
semi-global and local alignment types of Sec. II, and the sum-of-pairs score with affine gaps
(natural gap costs; the paper's future work, Sec. VI) with its textbook pairwise counterpart.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. The product library never loads it, and it shares no code with the CUDA path.

Residues are integer codes ``0..K-1`` (numpy uint8); in alignment rows a gap is ``GAP`` (255).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

GAP = 255
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``liboracle.so`` next to it (plain g++, -O2)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", _SRC,
                                   "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.oracle_align.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, u8p, ctypes.c_int,
                                     ctypes.c_int, i32p, ctypes.c_int32, i64p, u8p,
                                     ctypes.c_int64, i64p]
        lib.oracle_align.restype = ctypes.c_int
        lib.oracle_sp_score.argtypes = [u8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, i32p,
                                        ctypes.c_int32, i64p]
        lib.oracle_sp_score.restype = ctypes.c_int
        lib.oracle_nw2.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, ctypes.c_int, i32p,
                                   ctypes.c_int32, i64p]
        lib.oracle_nw2.restype = ctypes.c_int
        lib.oracle_align_many.argtypes = [u8p, i64p, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_int64, ctypes.c_int, i32p, ctypes.c_int32,
                                          i64p]
        lib.oracle_align_many.restype = ctypes.c_int
        lib.oracle_align_many_mt.argtypes = [u8p, i64p, ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_int64, ctypes.c_int, i32p, ctypes.c_int32,
                                             i64p, ctypes.c_int]
        lib.oracle_align_many_mt.restype = ctypes.c_int
        lib.oracle_align_type.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, u8p, ctypes.c_int,
                                          ctypes.c_int, i32p, ctypes.c_int32, ctypes.c_int, i64p]
        lib.oracle_align_type.restype = ctypes.c_int
        lib.oracle_align_type_tb.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, u8p,
                                             ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32,
                                             ctypes.c_int, i64p, u8p, ctypes.c_int64, i64p, i32p,
                                             i32p]
        lib.oracle_align_type_tb.restype = ctypes.c_int
        lib.oracle_align_affine.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, u8p,
                                            ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32,
                                            ctypes.c_int32, i64p, u8p, ctypes.c_int64, i64p]
        lib.oracle_align_affine.restype = ctypes.c_int
        lib.oracle_gotoh2.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_int, ctypes.c_int, i32p,
                                      ctypes.c_int32, ctypes.c_int32, i64p]
        lib.oracle_gotoh2.restype = ctypes.c_int
        _lib = lib
    return _lib


def _u8(x) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)  # valid pointer for empty sequences
    return a


def _sub(sub) -> tuple[np.ndarray, int]:
    s = np.ascontiguousarray(np.asarray(sub, dtype=np.int32))
    if s.ndim != 2 or s.shape[0] != s.shape[1]:
        raise ValueError("substitution matrix must be K x K")
    return s, int(s.shape[0])


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def align(s0, s1, s2, sub, gap: int, traceback: bool = False):
    """Optimal global 3-way SP score; with ``traceback`` also the (3, L) alignment (gap = 255).

    Returns ``score`` or ``(score, rows)``.
    """
    lib = _load()
    n = [len(s0), len(s1), len(s2)]
    a0, a1, a2 = _u8(s0), _u8(s1), _u8(s2)
    sm, K = _sub(sub)
    score = ctypes.c_int64(0)
    if traceback:
        cap = max(1, sum(n))
        rows = np.zeros(3 * cap, dtype=np.uint8)
        L = ctypes.c_int64(0)
        rc = lib.oracle_align(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8), n[1],
                              _ptr(a2, ctypes.c_uint8), n[2], K, _ptr(sm, ctypes.c_int32),
                              int(gap), ctypes.byref(score), _ptr(rows, ctypes.c_uint8), cap,
                              ctypes.byref(L))
        if rc:
            raise RuntimeError(f"oracle_align failed ({rc})")
        r = rows.reshape(3, cap)[:, : L.value].copy()
        return int(score.value), r
    rc = lib.oracle_align(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8), n[1],
                          _ptr(a2, ctypes.c_uint8), n[2], K, _ptr(sm, ctypes.c_int32), int(gap),
                          ctypes.byref(score), None, 0, None)
    if rc:
        raise RuntimeError(f"oracle_align failed ({rc})")
    return int(score.value)


def sp_score(rows, sub, gap: int) -> int:
    """Sum-of-pairs score of a (3, L) alignment (gap = 255)."""
    lib = _load()
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.uint8))
    if r.ndim != 2 or r.shape[0] != 3:
        raise ValueError("rows must be (3, L)")
    L = r.shape[1]
    buf = r if L else np.zeros((3, 1), dtype=np.uint8)
    sm, K = _sub(sub)
    out = ctypes.c_int64(0)
    rc = lib.oracle_sp_score(_ptr(buf, ctypes.c_uint8), L, buf.shape[1], K,
                             _ptr(sm, ctypes.c_int32), int(gap), ctypes.byref(out))
    if rc:
        raise ValueError("residue code out of range")
    return int(out.value)


def nw2(x, y, sub, gap: int) -> int:
    """Pairwise Needleman-Wunsch score with a linear gap (alpha per residue-gap pair)."""
    lib = _load()
    ax, ay = _u8(x), _u8(y)
    sm, K = _sub(sub)
    out = ctypes.c_int64(0)
    lib.oracle_nw2(_ptr(ax, ctypes.c_uint8), len(x), _ptr(ay, ctypes.c_uint8), len(y), K,
                   _ptr(sm, ctypes.c_int32), int(gap), ctypes.byref(out))
    return int(out.value)


def align_many(triplets, sub, gap: int, threads: int = 1) -> np.ndarray:
    """Scores (int64) of a list of (s0, s1, s2) triplets: one after another on one core, or
    spread over `threads` host threads (independent triplets, the same per-triplet DP)."""
    lib = _load()
    seqs = [np.asarray(s, dtype=np.uint8) for t in triplets for s in t]
    lens = np.array([len(s) for s in seqs], dtype=np.int32)
    offs = np.zeros(len(seqs), dtype=np.int64)
    if len(seqs):
        offs[1:] = np.cumsum(lens[:-1])
    codes = _u8(np.concatenate(seqs) if seqs else [])
    sm, K = _sub(sub)
    out = np.zeros(len(triplets), dtype=np.int64)
    if threads > 1:
        rc = lib.oracle_align_many_mt(_ptr(codes, ctypes.c_uint8), _ptr(offs, ctypes.c_int64),
                                      _ptr(lens, ctypes.c_int32), len(triplets), K,
                                      _ptr(sm, ctypes.c_int32), int(gap),
                                      _ptr(out, ctypes.c_int64), int(threads))
    else:
        rc = lib.oracle_align_many(_ptr(codes, ctypes.c_uint8), _ptr(offs, ctypes.c_int64),
                                   _ptr(lens, ctypes.c_int32), len(triplets), K,
                                   _ptr(sm, ctypes.c_int32), int(gap), _ptr(out, ctypes.c_int64))
    if rc:
        raise RuntimeError(f"oracle_align_many failed ({rc})")
    return out


GLOBAL, SEMIGLOBAL, LOCAL = 0, 1, 2


def align_type(s0, s1, s2, sub, gap: int, kind: int) -> int:
    """Score of the alignment type ``kind`` of Sec. II: GLOBAL (M[a][b][c]), SEMIGLOBAL (zero
    axes, best cell on a last slice) or LOCAL (zero axes, v = 0, best cell of the cube)."""
    lib = _load()
    n = [len(s0), len(s1), len(s2)]
    a0, a1, a2 = _u8(s0), _u8(s1), _u8(s2)
    sm, K = _sub(sub)
    score = ctypes.c_int64(0)
    rc = lib.oracle_align_type(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8), n[1],
                               _ptr(a2, ctypes.c_uint8), n[2], K, _ptr(sm, ctypes.c_int32),
                               int(gap), int(kind), ctypes.byref(score))
    if rc:
        raise RuntimeError(f"oracle_align_type failed ({rc})")
    return int(score.value)


def align_type_tb(s0, s1, s2, sub, gap: int, kind: int):
    """(score, rows (3, L), begin (i0, j0, k0), end (i1, j1, k1)) of the alignment type ``kind``:
    the rows align S0[i0:i1], S1[j0:j1], S2[k0:k1]. End cell: the first cell in (i, j, k) order
    with the best score among those that count; walk: first maximal move in Eq. 1's order, v
    last; stops at axis cells and, for LOCAL, where v = 0 alone is maximal."""
    lib = _load()
    n = [len(s0), len(s1), len(s2)]
    a0, a1, a2 = _u8(s0), _u8(s1), _u8(s2)
    sm, K = _sub(sub)
    cap = max(1, sum(n))
    rows = np.zeros(3 * cap, dtype=np.uint8)
    score, L = ctypes.c_int64(0), ctypes.c_int64(0)
    beg, end = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
    rc = lib.oracle_align_type_tb(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8), n[1],
                                  _ptr(a2, ctypes.c_uint8), n[2], K, _ptr(sm, ctypes.c_int32),
                                  int(gap), int(kind), ctypes.byref(score),
                                  _ptr(rows, ctypes.c_uint8), cap, ctypes.byref(L), beg, end)
    if rc:
        raise RuntimeError(f"oracle_align_type_tb failed ({rc})")
    r = rows.reshape(3, cap)[:, : L.value].copy()
    return int(score.value), r, tuple(beg), tuple(end)


def align_affine(s0, s1, s2, sub, gap: int, gap_open: int, traceback: bool = False):
    """Global 3-way score under affine gaps with natural gap costs: the sum over the three pairs
    of the induced pairwise alignment's score (columns with a gap in both sequences of the pair
    deleted), sigma per residue pair, `gap` per residue against a gap and `gap_open` per maximal
    gap run. With gap_open = 0 it equals align(). With ``traceback`` also the (3, L) rows.
    (The paper names affine gaps as future work, Sec. VI; this definition is the build's reading.)"""
    lib = _load()
    n = [len(s0), len(s1), len(s2)]
    a0, a1, a2 = _u8(s0), _u8(s1), _u8(s2)
    sm, K = _sub(sub)
    score = ctypes.c_int64(0)
    if traceback:
        cap = max(1, sum(n))
        rows = np.zeros(3 * cap, dtype=np.uint8)
        L = ctypes.c_int64(0)
        rc = lib.oracle_align_affine(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8),
                                     n[1], _ptr(a2, ctypes.c_uint8), n[2], K,
                                     _ptr(sm, ctypes.c_int32), int(gap), int(gap_open),
                                     ctypes.byref(score), _ptr(rows, ctypes.c_uint8), cap,
                                     ctypes.byref(L))
        if rc:
            raise RuntimeError(f"oracle_align_affine failed ({rc})")
        return int(score.value), rows.reshape(3, cap)[:, : L.value].copy()
    rc = lib.oracle_align_affine(_ptr(a0, ctypes.c_uint8), n[0], _ptr(a1, ctypes.c_uint8), n[1],
                                 _ptr(a2, ctypes.c_uint8), n[2], K, _ptr(sm, ctypes.c_int32),
                                 int(gap), int(gap_open), ctypes.byref(score), None, 0, None)
    if rc:
        raise RuntimeError(f"oracle_align_affine failed ({rc})")
    return int(score.value)


def gotoh2(x, y, sub, gap: int, gap_open: int) -> int:
    """Textbook pairwise alignment score with affine gaps (a gap run of length l scores
    gap_open + l * gap)."""
    lib = _load()
    ax, ay = _u8(x), _u8(y)
    sm, K = _sub(sub)
    out = ctypes.c_int64(0)
    lib.oracle_gotoh2(_ptr(ax, ctypes.c_uint8), len(x), _ptr(ay, ctypes.c_uint8), len(y), K,
                      _ptr(sm, ctypes.c_int32), int(gap), int(gap_open), ctypes.byref(out))
    return int(out.value)
