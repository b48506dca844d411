"""Thin ctypes binding of include/trioseq.h (argument marshalling only).

Every function named ``trioseq_*`` here calls the C entry point of the same name; all alignment
work happens in the CUDA library. If the library cannot be loaded the import raises — there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import itertools
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, EAGAIN, EOVERFLOW, ETIMEOUT, ECUDA, ENOTIMPL, ESCRATCH = range(9)
SCORE_ONLY, WITH_TRACEBACK = 0, 1
GLOBAL, SEMIGLOBAL, LOCAL = 0, 1, 2  # alignment types of Sec. II (trioseq_plan flags)
# trioseq_partition schemes: the three of Sec. V-D, and the dynamic rule taken largest first
PART_BLOCKED, PART_INTERLEAVED, PART_DYNAMIC, PART_LARGEST_FIRST = 0, 1, 2, 3


class TrioseqError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {trioseq_strerror(status)} ({status})")
        self.status = status


class Scoring(ctypes.Structure):
    _fields_ = [("alphabet", ctypes.c_char_p), ("alphabet_size", ctypes.c_int32),
                ("sub", ctypes.POINTER(ctypes.c_int8)), ("gap", ctypes.c_int32)]


class Triplet(ctypes.Structure):
    _fields_ = [("s", ctypes.c_char_p * 3), ("len", ctypes.c_uint32 * 3)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building first if needed) the engine library."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"engine library missing: {_build.LIB} (run build())")
    lib = ctypes.CDLL(_build.LIB)
    vp, sz, u32, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_int32
    i32p = ctypes.POINTER(ctypes.c_int32)
    szp = ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "trioseq_plan": ([ctypes.POINTER(Scoring), u32, u32, ctypes.POINTER(vp)], i32),
        "trioseq_plan_destroy": ([vp], i32),
        "trioseq_align_batch": ([vp, ctypes.POINTER(Triplet), sz, u32, i32p, vp], i32),
        "trioseq_traceback": ([vp, sz, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p, sz,
                               szp], i32),
        "trioseq_batch_create": ([vp, ctypes.POINTER(Triplet), sz, u32, ctypes.POINTER(vp)], i32),
        "trioseq_batch_run": ([vp, vp], i32),
        "trioseq_batch_scores": ([vp, vp, i32p], i32),
        "trioseq_batch_device_scores": ([vp, ctypes.POINTER(vp)], i32),
        "trioseq_batch_alignment": ([vp, sz, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p,
                                     sz, szp], i32),
        "trioseq_batch_info": ([vp, szp, ctypes.POINTER(ctypes.c_uint64),
                                ctypes.POINTER(ctypes.c_uint64), i32p, i32p], i32),
        "trioseq_batch_destroy": ([vp], i32),
        "trioseq_batch_profile": ([vp, i32], i32),
        "trioseq_batch_timing": ([vp, ctypes.POINTER(ctypes.c_float)], i32),
        "trioseq_plan_io_bytes": ([vp, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_uint64)], i32),
        "trioseq_server_create": ([ctypes.POINTER(vp), i32, sz, ctypes.POINTER(vp)], i32),
        "trioseq_submit": ([vp, ctypes.POINTER(Triplet), i32, u32,
                            ctypes.POINTER(ctypes.c_uint64)], i32),
        "trioseq_poll": ([vp, ctypes.c_uint64, i32p, ctypes.POINTER(ctypes.c_char_p), sz, szp],
                         i32),
        "trioseq_server_destroy": ([vp], i32),
        "trioseq_strerror": ([i32], ctypes.c_char_p),
        "trioseq_align_noalloc": ([ctypes.POINTER(Scoring), vp, u32, vp, u32, vp, u32, vp, vp],
                                  i32),
        "trioseq_plan_autotune": ([vp, ctypes.POINTER(Triplet), sz, u32, i32p, i32p, i32p], i32),
        "trioseq_batch_packing": ([vp, i32p], i32),
        "trioseq_batch_kernel": ([vp, ctypes.c_char_p, sz], i32),
        "trioseq_plan_affine": ([ctypes.POINTER(Scoring), i32, u32, ctypes.POINTER(vp)], i32),
        "trioseq_batch_slabs": ([vp, i32p, i32p], i32),
        "trioseq_traceback_span": ([vp, sz, i32p, i32p], i32),
        "trioseq_batch_span": ([vp, sz, i32p, i32p], i32),
        "trioseq_alu_rate": ([i32, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)], i32),
        "trioseq_partition": ([ctypes.POINTER(ctypes.c_uint32), sz, i32, i32, i32p,
                               ctypes.POINTER(ctypes.c_uint64)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return ["trioseq_plan", "trioseq_plan_destroy", "trioseq_align_batch", "trioseq_traceback",
            "trioseq_batch_create", "trioseq_batch_run", "trioseq_batch_scores",
            "trioseq_batch_device_scores", "trioseq_batch_alignment", "trioseq_batch_info",
            "trioseq_batch_destroy", "trioseq_batch_profile", "trioseq_batch_timing",
            "trioseq_plan_io_bytes", "trioseq_server_create", "trioseq_submit", "trioseq_poll",
            "trioseq_server_destroy", "trioseq_strerror", "trioseq_align_noalloc",
            "trioseq_plan_autotune", "trioseq_batch_packing", "trioseq_batch_kernel",
            "trioseq_plan_affine",
            "trioseq_batch_slabs",
            "trioseq_traceback_span", "trioseq_batch_span", "trioseq_alu_rate",
            "trioseq_partition"]


def trioseq_partition(lens, nranks: int, scheme: int = None):
    """Ranks of a triplet set under a Sec. V-D scheme (default dynamic), from an (n, 3) array of
    lengths. Returns (rank_of as an int32 array of n, cells per rank as a uint64 array)."""
    scheme = PART_DYNAMIC if scheme is None else scheme
    lens = np.ascontiguousarray(np.asarray(lens, dtype=np.uint32).reshape(-1, 3))
    n = lens.shape[0]
    rank_of = np.zeros(n, dtype=np.int32)
    load_ = np.zeros(max(int(nranks), 0), dtype=np.uint64)
    _check(load().trioseq_partition(
        lens.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), n, int(nranks), int(scheme),
        rank_of.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        load_.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if load_.size else None),
        "trioseq_partition")
    return rank_of, load_


def trioseq_plan_autotune(plan, sample, mode: int = SCORE_ONLY) -> dict:
    """Measure the kernel variants on `sample` and remember the fastest for its class."""
    arr, keep = _triplet_array(sample)
    tj, tk, ti = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().trioseq_plan_autotune(plan, arr, len(sample), int(mode), ctypes.byref(tj),
                                        ctypes.byref(tk), ctypes.byref(ti)),
           "trioseq_plan_autotune")
    del keep
    return {"tile": (tj.value, tk.value), "ti": ti.value}


def trioseq_strerror(status: int) -> str:
    return load().trioseq_strerror(int(status)).decode()


def _check(st: int, what: str):
    if st != OK:
        raise TrioseqError(st, what)


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _as_bytes(s) -> bytes:
    if isinstance(s, bytes):
        return s
    if isinstance(s, str):
        return s.encode()
    return bytes(np.asarray(s, dtype=np.uint8))


_TRIPLET_DTYPE = np.dtype({"names": ["s", "len"], "formats": [("<u8", 3), ("<u4", 3)],
                           "offsets": [Triplet.s.offset, Triplet.len.offset],
                           "itemsize": ctypes.sizeof(Triplet)})


def _triplet_array(triplets):
    """Triplet records (as a ctypes pointer) plus the objects keeping the strings alive.

    All sequences are joined into one bytes object and the records, filled with numpy, point
    into it, so marshalling thousands of triplets costs one copy of the residues rather than one
    Python call per field. The library only reads the strings (it copies them before returning)."""
    n = len(triplets)
    if any(len(t) != 3 for t in triplets):
        raise ValueError("a triplet has three sequences")
    flat = list(itertools.chain.from_iterable(triplets))
    try:  # all str (the common case): one join, one byte per character, as residues are
        joined = "".join(flat).encode("latin-1")
        lens = np.fromiter(map(len, flat), dtype=np.uint32, count=3 * n)
    except TypeError:  # bytes or code arrays among them
        parts = [_as_bytes(x) for x in flat]
        lens = np.fromiter(map(len, parts), dtype=np.uint32, count=3 * n)
        joined = b"".join(parts)
    base = ctypes.c_char_p(joined)  # points into the bytes object, which `keep` holds alive
    offs = np.zeros(3 * n, dtype=np.uint64)
    if n:
        offs[1:] = np.cumsum(lens[:-1], dtype=np.uint64)
    rec = np.zeros(max(1, n), dtype=_TRIPLET_DTYPE)
    addr = ctypes.cast(base, ctypes.c_void_p).value or 0
    rec["s"][:n] = (np.uint64(addr) + offs).reshape(n, 3)
    rec["len"][:n] = lens.reshape(n, 3)
    return rec.ctypes.data_as(ctypes.POINTER(Triplet)), (joined, base, rec)


def trioseq_plan(alphabet: str, sub, gap: int, flags: int = 0):
    """Plan for one scoring scheme; ``flags`` is the alignment type (GLOBAL, SEMIGLOBAL, LOCAL)."""
    lib = load()
    sub = np.ascontiguousarray(np.asarray(sub, dtype=np.int8))
    K = len(alphabet)
    if sub.shape != (K, K):
        raise ValueError("substitution matrix must be K x K")
    sc = Scoring(alphabet.encode(), K, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(gap))
    h = ctypes.c_void_p()
    _check(lib.trioseq_plan(ctypes.byref(sc), 0, int(flags), ctypes.byref(h)), "trioseq_plan")
    return h


def trioseq_plan_affine(alphabet: str, sub, gap: int, gap_open: int, flags: int = 0):
    """Plan for the sum-of-pairs score with affine gaps (natural gap costs): ``gap`` per residue
    against a gap, ``gap_open`` per maximal gap run of a pair. Score only, global type."""
    lib = load()
    sub = np.ascontiguousarray(np.asarray(sub, dtype=np.int8))
    K = len(alphabet)
    if sub.shape != (K, K):
        raise ValueError("substitution matrix must be K x K")
    sc = Scoring(alphabet.encode(), K, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(gap))
    h = ctypes.c_void_p()
    _check(lib.trioseq_plan_affine(ctypes.byref(sc), int(gap_open), int(flags), ctypes.byref(h)),
           "trioseq_plan_affine")
    return h


def trioseq_plan_destroy(plan):
    _check(load().trioseq_plan_destroy(plan), "trioseq_plan_destroy")


def trioseq_align_batch(plan, triplets, mode: int = SCORE_ONLY, stream=None) -> np.ndarray:
    lib = load()
    arr, keep = _triplet_array(triplets)
    out = np.zeros(max(1, len(triplets)), dtype=np.int32)
    _check(lib.trioseq_align_batch(plan, arr, len(triplets), int(mode),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   _stream_ptr(stream)), "trioseq_align_batch")
    del keep
    return out[:len(triplets)]


def _rows(fn, handle, idx: int, cap: int | None = None):
    lib = load()
    n = ctypes.c_size_t(0)
    st = fn(handle, idx, None, None, None, 0, ctypes.byref(n))  # size query
    if st == OK:
        return ("", "", "")
    if st != EINVAL or n.value == 0:
        _check(st, fn.__name__)
    cap = n.value if cap is None else cap
    bufs = [ctypes.create_string_buffer(max(1, cap)) for _ in range(3)]
    _check(fn(handle, idx, bufs[0], bufs[1], bufs[2], cap, ctypes.byref(n)), fn.__name__)
    return tuple(b.raw[:n.value].decode() for b in bufs)


def trioseq_traceback(plan, idx: int, cap: int | None = None):
    """Aligned rows (three strings, '-' = gap) of triplet idx of the last traceback batch."""
    return _rows(load().trioseq_traceback, plan, idx, cap)


def trioseq_batch_create(plan, triplets, mode: int = SCORE_ONLY):
    lib = load()
    arr, keep = _triplet_array(triplets)
    h = ctypes.c_void_p()
    _check(lib.trioseq_batch_create(plan, arr, len(triplets), int(mode), ctypes.byref(h)),
           "trioseq_batch_create")
    del keep
    return h


def trioseq_batch_run(batch, stream=None):
    _check(load().trioseq_batch_run(batch, _stream_ptr(stream)), "trioseq_batch_run")


def trioseq_batch_scores(batch, n: int, stream=None) -> np.ndarray:
    out = np.zeros(max(1, n), dtype=np.int32)
    _check(load().trioseq_batch_scores(batch, _stream_ptr(stream),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "trioseq_batch_scores")
    return out[:n]


def trioseq_batch_device_scores(batch) -> int:
    p = ctypes.c_void_p()
    _check(load().trioseq_batch_device_scores(batch, ctypes.byref(p)),
           "trioseq_batch_device_scores")
    return p.value or 0


def trioseq_batch_alignment(batch, idx: int, cap: int | None = None):
    return _rows(load().trioseq_batch_alignment, batch, idx, cap)


def _span(fn, handle, idx: int):
    beg, end = (ctypes.c_int32 * 3)(), (ctypes.c_int32 * 3)()
    _check(fn(handle, idx, beg, end), fn.__name__)
    return tuple(beg), tuple(end)


def trioseq_traceback_span(plan, idx: int):
    """((i0, j0, k0), (i1, j1, k1)): the rows of triplet idx align S0[i0:i1], S1[j0:j1], S2[k0:k1]."""
    return _span(load().trioseq_traceback_span, plan, idx)


def trioseq_batch_span(batch, idx: int):
    return _span(load().trioseq_batch_span, batch, idx)


def trioseq_batch_info(batch) -> dict:
    n = ctypes.c_size_t()
    cells, tasks = ctypes.c_uint64(), ctypes.c_uint64()
    tj, tk = ctypes.c_int32(), ctypes.c_int32()
    _check(load().trioseq_batch_info(batch, ctypes.byref(n), ctypes.byref(cells),
                                     ctypes.byref(tasks), ctypes.byref(tj), ctypes.byref(tk)),
           "trioseq_batch_info")
    per = ctypes.c_int32()
    _check(load().trioseq_batch_packing(batch, ctypes.byref(per)), "trioseq_batch_packing")
    sl, ns = ctypes.c_int32(), ctypes.c_int32()
    _check(load().trioseq_batch_slabs(batch, ctypes.byref(sl), ctypes.byref(ns)),
           "trioseq_batch_slabs")
    name = ctypes.create_string_buffer(160)
    _check(load().trioseq_batch_kernel(batch, name, 160), "trioseq_batch_kernel")
    kernel, _, label = name.value.decode().partition(" tile ")
    return {"n": n.value, "cells": cells.value, "tasks": tasks.value, "tile": (tj.value, tk.value),
            "packing": per.value, "slab_slices": sl.value, "slabs": ns.value, "kernel": kernel,
            "tile_label": label}


def trioseq_batch_destroy(batch):
    _check(load().trioseq_batch_destroy(batch), "trioseq_batch_destroy")


def trioseq_batch_profile(batch, enable: bool = True):
    _check(load().trioseq_batch_profile(batch, int(bool(enable))), "trioseq_batch_profile")


def trioseq_batch_timing(batch) -> tuple[float, float]:
    """(wavefront kernel ms, walk ms) of the last profiled run."""
    ms = (ctypes.c_float * 2)()
    _check(load().trioseq_batch_timing(batch, ms), "trioseq_batch_timing")
    return float(ms[0]), float(ms[1])


def trioseq_plan_io_bytes(plan) -> tuple[int, int]:
    h2d, d2h = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().trioseq_plan_io_bytes(plan, ctypes.byref(h2d), ctypes.byref(d2h)),
           "trioseq_plan_io_bytes")
    return h2d.value, d2h.value


def trioseq_server_create(plans, hbm_budget: int = 0):
    arr = (ctypes.c_void_p * len(plans))(*[p.value if hasattr(p, "value") else p for p in plans])
    h = ctypes.c_void_p()
    _check(load().trioseq_server_create(arr, len(plans), int(hbm_budget), ctypes.byref(h)),
           "trioseq_server_create")
    return h


def trioseq_submit(server, triplet, plan_id: int, mode: int = SCORE_ONLY):
    """Returns (status, ticket); status is OK or EAGAIN (queue full)."""
    arr, keep = _triplet_array([triplet])
    t = ctypes.c_uint64(0)
    st = load().trioseq_submit(server, arr, int(plan_id), int(mode), ctypes.byref(t))
    if st not in (OK, EAGAIN):
        _check(st, "trioseq_submit")
    return st, t.value


def trioseq_poll(server, ticket: int, cap: int = 0):
    """Returns (status, score, rows or None); status is OK or EAGAIN."""
    score = ctypes.c_int32(0)
    n = ctypes.c_size_t(0)
    if cap > 0:
        bufs = [ctypes.create_string_buffer(cap) for _ in range(3)]
        rows = (ctypes.c_char_p * 3)(*[ctypes.cast(b, ctypes.c_char_p) for b in bufs])
    else:
        bufs, rows = None, None
    st = load().trioseq_poll(server, ctypes.c_uint64(ticket), ctypes.byref(score), rows,
                             int(cap), ctypes.byref(n))
    if st == EAGAIN:
        return st, None, None
    _check(st, "trioseq_poll")
    out_rows = tuple(b.raw[:n.value].decode() for b in bufs) if bufs and n.value else None
    return st, int(score.value), out_rows


def trioseq_server_destroy(server):
    _check(load().trioseq_server_destroy(server), "trioseq_server_destroy")


ALU_FORMS = ("max", "add_max", "max3", "add3", "mad_by_one")  # trioseq_alu_rate's op codes


def trioseq_alu_rate(op: int) -> tuple[float, float]:
    """(instructions per SM clock per SM, SM MHz) of int32 instruction form `op` (ALU_FORMS)."""
    rate, mhz = ctypes.c_double(0), ctypes.c_double(0)
    _check(load().trioseq_alu_rate(int(op), ctypes.byref(rate), ctypes.byref(mhz)),
           "trioseq_alu_rate")
    return rate.value, mhz.value


def trioseq_align_noalloc(alphabet: str, sub, gap: int, d_s0: int, a: int, d_s1: int, b: int,
                          d_s2: int, c: int, d_score: int, stream=None) -> int:
    """Allocation-free scoring of one triplet. d_s0/d_s1/d_s2 are device addresses of the raw
    sequence bytes, d_score the device address of one int32. Returns the status code (OK on
    success; errors are returned, not raised, so callers can test ESCRATCH)."""
    sub = np.ascontiguousarray(np.asarray(sub, dtype=np.int8))
    sc = Scoring(alphabet.encode(), len(alphabet),
                 sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(gap))
    return int(load().trioseq_align_noalloc(ctypes.byref(sc), ctypes.c_void_p(d_s0 or None), a,
                                            ctypes.c_void_p(d_s1 or None), b,
                                            ctypes.c_void_p(d_s2 or None), c,
                                            ctypes.c_void_p(d_score), _stream_ptr(stream)))
