"""Stored full-size expected values (written by ``make_goldens.py`` from the oracle alone).

Readers for the golden files of the five workloads' large configurations, and the input digest
that ties each stored value to the exact seeded input it was computed on. If the generators in
``synth.py`` ever change, the digest no longer matches and the tests say so instead of comparing
against a value computed on other inputs.

No value here comes from the CUDA path: every score and alignment digest was computed by
``oracle/`` (Eq. 1 of Sec. II, global initialisation, first-maximal-move tie-break in Eq. 1's
listing order) on the inputs that ``synth.py`` generates.
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CONFIG0 = os.path.join(HERE, "config0_alignment.tsv")
CONFIG1 = os.path.join(HERE, "config1_alignment.tsv")
CONFIG2 = os.path.join(HERE, "config2_scores.tsv")
CONFIG3 = os.path.join(HERE, "config3_score.tsv")
CONFIG4 = os.path.join(HERE, "config4_sample.tsv")
CONFIG2_AFFINE = os.path.join(HERE, "config2_affine_first64.tsv")
AFFINE_SAMPLE = 64    # the first triplets of the config-2 batch, affine model
AFFINE_GAP_OPEN = -4  # gamma of the affine line (DNA scheme: alpha = -2 per residue)
CONFIG4_SAMPLE = 200  # the first requests of the serving stream (seed 1004)


def input_digest(triplets) -> str:
    """sha256 over every triplet's three lengths (uint32 little-endian) and residue codes."""
    h = hashlib.sha256()
    for t in triplets:
        for s in t:
            s = np.ascontiguousarray(np.asarray(s, dtype=np.uint8))
            h.update(np.uint32(len(s)).tobytes())
            h.update(s.tobytes())
    return h.hexdigest()


def rows_digest(rows_text) -> str:
    """sha256 of an alignment given as three text rows ('-' for a gap), joined by newlines."""
    return hashlib.sha256("\n".join(rows_text).encode()).hexdigest()


def _header(path):
    meta = {}
    with open(path) as f:
        for line in f:
            if not line.startswith("#"):
                break
            if line.startswith("#@"):
                k, v = line[2:].strip().split("=", 1)
                meta[k.strip()] = v.strip()
    return meta


def _rows(path):
    with open(path) as f:
        return [ln.rstrip("\n").split("\t") for ln in f if ln.strip() and not ln.startswith("#")]


def _load_alignment(path):
    rows = _rows(path)
    assert len(rows) == 1
    r = rows[0]
    return _header(path), {"score": int(r[0]), "aln_len": int(r[1]), "rows_sha256": r[2]}


def load_config0():
    """(meta, {score, aln_len, rows_sha256}) of the independent DNA triplet, 128 each."""
    return _load_alignment(CONFIG0)


def load_config1():
    """(meta, {score, aln_len, rows_sha256}) of the related DNA triplet, ancestor 1000."""
    return _load_alignment(CONFIG1)


def load_config2():
    """(meta, scores as an int64 array in batch order)."""
    rows = _rows(CONFIG2)
    scores = np.array([int(r[1]) for r in rows], dtype=np.int64)
    assert [int(r[0]) for r in rows] == list(range(len(rows)))
    return _header(CONFIG2), scores


def load_config2_affine():
    """(meta, scores of the first AFFINE_SAMPLE config-2 triplets under affine gaps)."""
    rows = _rows(CONFIG2_AFFINE)
    assert [int(r[0]) for r in rows] == list(range(len(rows)))
    return _header(CONFIG2_AFFINE), np.array([int(r[1]) for r in rows], dtype=np.int64)


def load_config3():
    """(meta, score)."""
    rows = _rows(CONFIG3)
    assert len(rows) == 1
    return _header(CONFIG3), int(rows[0][0])


def load_config4():
    """(meta, list of dicts: id, protein, traceback, lens, score, aln_len, rows_sha256)."""
    out = []
    for r in _rows(CONFIG4):
        out.append({"id": int(r[0]), "protein": r[1] == "1", "traceback": r[2] == "1",
                    "lens": tuple(int(x) for x in r[3].split(",")), "score": int(r[4]),
                    "aln_len": int(r[5]) if r[5] != "." else None,
                    "rows_sha256": r[6] if r[6] != "." else None})
    return _header(CONFIG4), out
