"""Write the full-size golden files from the oracle alone (test infrastructure).

    python tests/golden/make_goldens.py [--only c0,c1,c2,c2a,c3,c4] [--threads N]

Every stored value is computed by ``oracle/`` (plain int64 Eq. 1 of Sec. II with the global
initialisation and the first-maximal-move tie-break in Eq. 1's listing order) on the seeded
inputs of ``paper_2605_28400_gb300/synth.py``; nothing here touches the CUDA library.

- config0_alignment.tsv, config1_alignment.tsv: score, alignment length and the sha256 of the
  alignment's rows of the independent DNA triplet (128 each, seed 1000) and of the related DNA
  triplet (ancestor 1000, seed 1001).
- config2_scores.tsv: all 4,096 scores of the batch of related DNA triplets (ancestor lengths
  uniform in [100, 300], seed 1002), independent triplets spread over host threads.
- config2_affine_first64.tsv: the first 64 triplets of that batch under affine gaps (natural
  gap costs, alpha = -2, gamma = -4; the build's reading of the paper's future work, Sec. VI).
- config3_score.tsv: the score of the protein triplet with ancestor length 4000 (seed 1003),
  about 6.4e10 cells on one host core.
- config4_sample.tsv: the first 200 requests of the serving stream (seed 1004: 70% DNA, 30%
  protein, ancestor lengths lognormal(ln 300, 0.8) clipped to [50, 2000], 20% with traceback):
  every score, and for traceback requests the alignment's length and the sha256 of its rows.

Each file records the digest of the inputs it was computed on (``goldens.input_digest``).
"""
from __future__ import annotations

import argparse
import os
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2605_28400_gb300 import synth  # noqa: E402
from tests.golden import goldens  # noqa: E402

CITE = ("# Expected values of the exact 3-way global alignment: Eq. 1 (Sec. II) with the SOP column\n"
        "# score and the global initialisation of Sec. II, first maximal move in Eq. 1's listing order.\n"
        "# Computed by the oracle (oracle/oracle.cpp, int64) on the seeded synthetic inputs of\n"
        "# paper_2605_28400_gb300/synth.py; written by tests/golden/make_goldens.py.\n")


def _write(path, lines, meta, desc):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write(CITE)
        f.write(desc)
        for k, v in meta.items():
            f.write(f"#@ {k} = {v}\n")
        for ln in lines:
            f.write(ln + "\n")
    os.replace(tmp, path)


def _text_rows(rows, sc):
    return ["".join("-" if v == oracle.GAP else sc.alphabet[v] for v in row) for row in rows]


def make_alignment(which):
    w, seed, path, desc = {
        "c0": (synth.config0(), 1000, goldens.CONFIG0,
               "# Config 0: three independent uniform ACGT sequences of length 128.\n"),
        "c1": (synth.config1(), 1001, goldens.CONFIG1,
               "# Config 1: related DNA triplet, ancestor 1000, 5% subs, 2% indels (mean 2).\n"),
    }[which]
    t0 = time.time()
    score, rows = oracle.align(*w.triplets[0], w.scoring.sub, w.scoring.gap, traceback=True)
    dt = time.time() - t0
    meta = {"workload": w.name, "seed": seed, "lens": ",".join(str(len(s)) for s in w.triplets[0]),
            "cells": w.cells, "input_sha256": goldens.input_digest(w.triplets),
            "oracle_seconds": f"{dt:.1f} on 1 thread"}
    _write(path, [f"{score}\t{rows.shape[1]}\t{goldens.rows_digest(_text_rows(rows, w.scoring))}"],
           meta, desc + "# Columns: score, alignment length, sha256 of the three text rows ('-' = gap)\n"
                        "# joined by newlines.\n")
    print(f"{which}: score {score}, {rows.shape[1]} columns in {dt:.1f} s", flush=True)


def make_config2(threads):
    w = synth.config2()
    t0 = time.time()
    scores = oracle.align_many(w.triplets, w.scoring.sub, w.scoring.gap, threads=threads)
    dt = time.time() - t0
    meta = {"workload": w.name, "seed": 1002, "triplets": len(w.triplets), "cells": w.cells,
            "input_sha256": goldens.input_digest(w.triplets),
            "oracle_seconds": f"{dt:.1f} on {threads} threads"}
    _write(goldens.CONFIG2, [f"{i}\t{int(s)}" for i, s in enumerate(scores)], meta,
           "# Config 2: 4096 related DNA triplets, ancestor U{100..300}, 5% subs, 2% indels (mean 2).\n"
           "# Columns: index in batch order, score.\n")
    print(f"config2: {len(scores)} scores in {dt:.1f} s", flush=True)


def make_config2_affine(threads):
    w = synth.config2()
    trips = w.triplets[:goldens.AFFINE_SAMPLE]
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        scores = list(ex.map(lambda t: oracle.align_affine(*t, w.scoring.sub, w.scoring.gap,
                                                           goldens.AFFINE_GAP_OPEN), trips))
    dt = time.time() - t0
    meta = {"workload": f"{w.name}, first {len(trips)}, affine", "seed": 1002,
            "gap_open": goldens.AFFINE_GAP_OPEN, "triplets": len(trips),
            "cells": sum(len(a) * len(b) * len(c) for a, b, c in trips),
            "input_sha256": goldens.input_digest(trips),
            "oracle_seconds": f"{dt:.1f} on {threads} threads"}
    _write(goldens.CONFIG2_AFFINE, [f"{i}\t{int(v)}" for i, v in enumerate(scores)], meta,
           "# Config 2 under affine gaps (natural gap costs: per pair, the induced alignment with its\n"
           "# all-gap columns deleted; alpha = -2 per residue against a gap, gamma = -4 per maximal\n"
           "# gap run): the first 64 triplets of the batch. Columns: index, score.\n")
    print(f"config2 affine: {len(scores)} scores in {dt:.1f} s", flush=True)


def make_config3():
    w = synth.config3()
    t0 = time.time()
    score = oracle.align(*w.triplets[0], w.scoring.sub, w.scoring.gap)
    dt = time.time() - t0
    meta = {"workload": w.name, "seed": 1003, "lens": ",".join(str(len(s)) for s in w.triplets[0]),
            "cells": w.cells, "input_sha256": goldens.input_digest(w.triplets),
            "oracle_seconds": f"{dt:.1f} on 1 thread"}
    _write(goldens.CONFIG3, [str(score)], meta,
           "# Config 3: protein triplet, ancestor 4000, 15% subs, 3% indels (mean 3), seeded\n"
           "# symmetric matrix (diagonal U{4..11}, off-diagonal U{-4..2}), gap -4.\n"
           "# Column: score.\n")
    print(f"config3: score {score} in {dt:.1f} s", flush=True)


def _one_request(args):
    r, dna, prot = args
    sc = prot if r["protein"] else dna
    t = r["triplet"]
    if not r["traceback"]:
        return oracle.align(*t, sc.sub, sc.gap), None, None
    score, rows = oracle.align(*t, sc.sub, sc.gap, traceback=True)
    return score, rows.shape[1], goldens.rows_digest(_text_rows(rows, sc))


def make_config4(threads):
    dna, prot, reqs = synth.config4(n=goldens.CONFIG4_SAMPLE)
    t0 = time.time()
    # largest first, so the long traceback cubes do not end up last on one thread
    order = sorted(range(len(reqs)),
                   key=lambda i: -len(reqs[i]["triplet"][0]) * len(reqs[i]["triplet"][1])
                   * len(reqs[i]["triplet"][2]))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = dict(zip(order, ex.map(_one_request, [(reqs[i], dna, prot) for i in order])))
    dt = time.time() - t0
    lines = []
    for i, r in enumerate(reqs):
        score, L, dig = res[i]
        lens = ",".join(str(len(s)) for s in r["triplet"])
        lines.append(f"{r['id']}\t{int(r['protein'])}\t{int(r['traceback'])}\t{lens}\t{score}\t"
                     f"{L if L is not None else '.'}\t{dig or '.'}")
    cells = sum(len(t[0]) * len(t[1]) * len(t[2]) for t in (r["triplet"] for r in reqs))
    meta = {"workload": f"serving_stream_first_{len(reqs)}", "seed": 1004, "requests": len(reqs),
            "cells": cells, "input_sha256": goldens.input_digest([r["triplet"] for r in reqs]),
            "oracle_seconds": f"{dt:.1f} on {threads} threads"}
    _write(goldens.CONFIG4, lines, meta,
           "# Config 4: first requests of the serving stream: 70% DNA (config-1 scoring), 30% protein\n"
           "# (config-3 scoring, matrix of seed 1004), ancestor lognormal(ln 300, 0.8) clipped to\n"
           "# [50, 2000], 20% with traceback.\n"
           "# Columns: id, protein, traceback, lengths, score, alignment length, sha256 of the three\n"
           "# text rows ('-' = gap) joined by newlines ('.' where no traceback is asked).\n")
    print(f"config4: {len(reqs)} requests in {dt:.1f} s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="c0,c1,c2,c2a,c3,c4")
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    which = set(a.only.split(","))
    oracle.build()
    # the long single-core config-3 run goes alongside the multi-threaded ones
    rest = max(1, a.threads - (1 if "c3" in which else 0))
    with ThreadPoolExecutor(max_workers=1) as ex:
        f3 = ex.submit(make_config3) if "c3" in which else None
        for c in ("c0", "c1"):
            if c in which:
                make_alignment(c)
        if "c2" in which:
            make_config2(rest)
        if "c2a" in which:
            make_config2_affine(rest)
        if "c4" in which:
            make_config4(rest)
        if f3 is not None:
            f3.result()


if __name__ == "__main__":
    main()
