#!/usr/bin/env python
"""Benchmark of the exact 3-way global alignment engine on GB300.

Metric: GCUPS = sum over triplets of |S0|*|S1|*|S2| / seconds / 1e9 (the paper's TCUPS
numerator, Sec. V-A, scaled to giga). One step = one full pass of the hot path over the
workload: workspace reset, the persistent wavefront kernel (all cells of Eq. 1, with the packed
traceback-code stream in traceback mode), and the traceback walk.

Default workload: the single-triplet, score-only case the roofline fraction is quoted on: one
related protein triplet, ancestor length 4000 with three descendants (15% substitutions, 3%
indels of geometric length, mean 3), seeded 20 x 20 substitution matrix, gap -4 (~6.4e10 cells).
The aux object adds the traceback workload (related DNA triplet, ancestor 1000, score + 4-bit
codes + walk), the 4096-triplet batch against one launch per triplet, and a serving stream with
p50/p99 latency.

value : device-resident inputs (uploaded once), CUDA events on the launching stream around each
        step, L2 flushed (256 MiB write) between timed steps outside the events.
e2e   : the public C call trioseq_align_batch on host strings per step (encode, H2D from pinned
        staging, kernels, D2H of scores and alignment), host wall clock.
roofline: the wavefront kernel's int32 work (13 algorithmic ops per cell: 7 adds + 6 max) over
        its own event-timed duration, against SMs x 128 int32 lanes x the median SM clock
        sampled during the timed region.
cpu_baseline / --impl reference: the C++ oracle (single core) on a bounded prefix sample.

Under torchrun (N > 1) the slowest rank's time is reported and `value` is the whole job's cells
over it (weak scaling; no collective on the data path). A batch workload (batch4096) becomes
N x 4096 triplets of the same recipe, sharded over the ranks by the dynamic partition of
Sec. V-D taken largest triplet first (trioseq_partition: least cumulative cells first), each
rank computing the same partition from the lengths. A single-triplet workload runs one replica per rank. The aux lines
and the CPU baseline are taken at N = 1 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GCUPS (3D cells/s) and % of INT32 roofline; batched vs per-triplet; p50/p99 lat"
OPS_PER_CELL = 13          # 7 adds + 6 max per cell (factored Eq. 1)
INT32_LANES_PER_SM = 128   # int32 ops/clk/SM: 64 fused add+max (VIADDMNMX) issues per clock per SM
# int32 operations per instruction of the forms that carry maxima. Maxima issue on the ALU pipe
# only; plain adds can also go to the FMA pipe (the add forms are measured and reported, but the
# max-plus roof is set by the forms with maxima).
ALU_OPS_PER_FORM = {"max": 1, "add_max": 2, "max3": 2}


def measured_alu(B) -> dict:
    """Issue rates of the cell update's int32 instruction forms on this GPU (trioseq_alu_rate,
    outside any timed region) and the int32 operations per SM per clock that the forms with
    maxima sustain: the best of operations-per-instruction x rate over those forms."""
    rates = {}
    for op, name in enumerate(B.ALU_FORMS):
        r, mhz = B.trioseq_alu_rate(op)
        rates[name] = {"per_clk_per_sm": r, "sm_mhz": mhz}
    lanes = max(ALU_OPS_PER_FORM[k] * rates[k]["per_clk_per_sm"] for k in ALU_OPS_PER_FORM)
    return {"forms": rates, "int32_ops_per_clk_per_sm": lanes}


def roof_lanes(alu: dict | None) -> float:
    """int32 lanes per SM per clock for the roofline: the lower of nominal and measured."""
    if not alu:
        return float(INT32_LANES_PER_SM)
    return min(float(INT32_LANES_PER_SM), alu["int32_ops_per_clk_per_sm"])
CODE_BYTES_PER_CELL = 0.5  # packed 4-bit traceback code


def workloads():
    from paper_2605_28400_gb300 import synth
    return {
        "dna1000": (synth.config1, "one related DNA triplet, ancestor 1000, 5% subs, 2% indels "
                                   "(geometric mean 2), +2/-1/-2, score + traceback"),
        "protein4000": (synth.config3, "one related protein triplet, ancestor 4000, 15% subs, "
                                       "3% indels (geometric mean 3), seeded 20x20 matrix, "
                                       "gap -4, score only"),
        "batch4096": (synth.config2, "4096 related DNA triplets, ancestor lengths U[100,300], "
                                     "score only, one persistent launch"),
        "dna128": (synth.config0, "one triplet of independent uniform DNA, 128 each, score + "
                                  "traceback"),
        # reduced-size case of the protein recipe (profiling captures that must stay small)
        "protein1000": (lambda: synth.config3(L=1000),
                        "one related protein triplet, ancestor 1000, protein recipe, score only"),
        "protein2000": (lambda: synth.config3(L=2000),
                        "one related protein triplet, ancestor 2000, protein recipe, score only"),
        # linear-space traceback: the 4-bit code cube (~256 GB) does not fit beside its records
        "dna8000": (lambda: synth.config1(L=8000),
                    "one related DNA triplet, ancestor 8000, config-1 recipe, score + traceback "
                    "in slabs (linear-space traceback)"),
    }


# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons, kept if taken inside [t0, t1]."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.samples = []
        self.proc = None
        self.thread = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True,
                bufsize=1)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            if self.uuid and self.uuid not in f[0]:
                continue
            self.samples.append((time.time(), f))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float) -> dict:
        inside = [f for (t, f) in self.samples if t0 <= t <= t1]
        note = "samples inside the timed region"
        if not inside and self.samples:
            inside = [min(self.samples, key=lambda s: abs(s[0] - 0.5 * (t0 + t1)))[1]]
            note = "nearest sample to the timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(f[1]) for f in inside if num(f[1])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for f in inside:
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": num(inside[0][2]), "reasons": sorted(reasons),
                "power_w_max": max((num(f[3]) or 0.0) for f in inside),
                "samples": len(inside), "note": note}


def kernel_source_hash(tile: str) -> str:
    """Hash of the sources a tile's wavefront kernel is compiled from: the two-cells-per-register
    kernel (tile 8x16, or a label ending in 'v', 's' or 't') or the int32 / two-triplets kernel
    family."""
    common = ("wavefront.cuh", "engine.h")
    own = (("wavefront_vl.cuh", "kernels_vl.cu") if tile.endswith(("v", "s", "t")) or tile == "8x16"
           else ("kernels.cu", "kernels_packed.cu", "kernels_slab.cu", "kernels_variants.cu"))
    h = hashlib.sha256()
    for f in common + own:
        with open(os.path.join(ROOT, "paper_2605_28400_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def global_workload(key: str, world: int):
    """The whole job's batch and its description when a multi-triplet workload runs on `world`
    ranks: `world` times the single-GPU batch (same recipe and seed), so each rank's share stays
    about the same size (weak scaling). (None, None) for single-triplet workloads, which run as
    replicas."""
    from paper_2605_28400_gb300 import synth
    if key == "batch4096":
        n = 4096 * world
        return synth.config2(n=n), (f"{n} related DNA triplets, ancestor lengths U[100,300], "
                                    f"score only, sharded over {world} ranks, one persistent "
                                    "launch per rank")
    return None, None


def shard_workload(w, world: int, rank: int, B):
    """This rank's share of a batch under the dynamic partition of Sec. V-D (each triplet to the
    rank with the least cumulative cells so far), taken largest triplet first. Every rank
    computes the same partition from the same lengths, so there is no collective. Returns
    (share, cells of every rank)."""
    from paper_2605_28400_gb300 import synth
    lens = [[len(s) for s in t] for t in w.triplets]
    rank_of, cells = B.trioseq_partition(lens, world, B.PART_LARGEST_FIRST)
    mine = [t for t, r in zip(w.triplets, rank_of) if r == rank]
    share = synth.Workload(f"{w.name}, rank {rank} of {world}", w.scoring, mine, w.traceback,
                           dict(w.meta))
    return share, [int(c) for c in cells]


def kernel_of(info: dict, n_triplets: int):
    """(tile label, kernel name) of a batch, as the library reports them (trioseq_batch_kernel):
    e.g. ("8x8v", "wavefront_vl_kernel<8,4,false>") for two column halves of one triplet per
    register, ("8x16s", ...) for its variant with the sigma''(y,z) tile in shared memory."""
    return info["tile_label"], info["kernel"]


def measured_traffic(key: str, tile: str):
    """DRAM bytes per launch of the wavefront kernel from the committed ncu summary, or None
    when the kernel source changed since the counters were taken or the batch runs another
    tile than the one measured."""
    path = os.path.join(ROOT, "profiles", "wavefront_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(f"{key}/{tile}") or d.get(key)  # per tile where several are measured
        if e and e.get("kernel_hash") == kernel_source_hash(tile) and e.get("tile") == tile:
            return e.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def triplet_strings(w):
    from paper_2605_28400_gb300 import synth
    return [[synth.to_str(s, w.scoring.alphabet) for s in t] for t in w.triplets]


def oracle_golden(key: str, w):
    """Stored oracle scores (and alignment digests) of a full-size workload, written by
    tests/golden/make_goldens.py from the oracle alone, or None when none is stored for it or
    the stored inputs' digest differs from this workload's inputs."""
    from tests.golden import goldens
    loaders = {"protein4000": goldens.load_config3, "batch4096": goldens.load_config2,
               "dna1000": goldens.load_config1, "dna128": goldens.load_config0}
    if key not in loaders:
        return None
    try:
        meta, want = loaders[key]()
    except (OSError, ValueError, AssertionError):
        return None
    if meta.get("input_sha256") != goldens.input_digest(w.triplets):
        return None
    return want


def check_golden(key: str, w, scores, rows=None):
    """True when the scores (and the rows of a one-triplet traceback workload) equal the stored
    oracle values, None when none are stored. A mismatch stops the benchmark: a number measured
    on wrong results is not reported."""
    from tests.golden import goldens
    want = oracle_golden(key, w)
    if want is None:
        return None
    if isinstance(want, dict):  # one triplet with its alignment
        ok = [int(x) for x in scores] == [want["score"]]
        if rows is not None:
            ok &= goldens.rows_digest(rows) == want["rows_sha256"]
    elif hasattr(want, "__len__"):
        ok = [int(x) for x in scores] == [int(x) for x in want]
    else:
        ok = [int(x) for x in scores] == [int(want)]
    assert ok, f"{key}: results differ from the stored oracle values"
    return True


# ------------------------------------------------------------------------------------------
def host_cpu() -> dict:
    """CPU model, logical core count and clock of the host running the oracle: the max MHz from
    lscpu, else cpufreq, else ACPI CPPC (nominal clock x highest / nominal performance); the
    current MHz of CPU 0 from cpufreq and the CPPC nominal MHz where the kernel exposes them."""
    model, max_mhz, cur_mhz = "", None, None
    try:  # lscpu names Arm cores (Neoverse-V2 on Grace); /proc/cpuinfo there does not
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            key = line.split(":", 1)[0].strip().lower()
            if key == "model name" and not model:
                model = line.split(":", 1)[1].strip()
            elif key == "cpu max mhz":
                try:
                    max_mhz = float(line.split(":", 1)[1].strip().replace(",", "."))
                except ValueError:
                    pass
    except (OSError, subprocess.SubprocessError):
        pass
    cpufreq = "/sys/devices/system/cpu/cpu0/cpufreq/"
    try:
        with open(cpufreq + "scaling_cur_freq") as fh:
            cur_mhz = int(fh.read().strip()) / 1000.0
    except (OSError, ValueError):
        pass
    if max_mhz is None:
        try:
            with open(cpufreq + "cpuinfo_max_freq") as fh:
                max_mhz = int(fh.read().strip()) / 1000.0
        except (OSError, ValueError):
            pass
    nominal_mhz = None
    cppc = "/sys/devices/system/cpu/cpu0/acpi_cppc/"
    try:  # Arm servers without cpufreq: ACPI CPPC gives the nominal clock and the perf range
        with open(cppc + "nominal_freq") as fh:
            nominal_mhz = float(fh.read().strip())
        if max_mhz is None:
            with open(cppc + "highest_perf") as fh, open(cppc + "nominal_perf") as gh:
                hi, nom = float(fh.read().strip()), float(gh.read().strip())
            if nom > 0:
                max_mhz = nominal_mhz * hi / nom
    except (OSError, ValueError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and not model:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu": model, "nproc": os.cpu_count(), "max_mhz": max_mhz, "cur_mhz": cur_mhz,
            "nominal_mhz": nominal_mhz, "measured_mhz": measured_host_mhz(),
            "measured_mhz_method": "one host thread: a dependent chain of n (add, xor) pairs, "
                                   "2 cycles per pair (1-cycle integer add and xor latency on "
                                   "x86-64 and Neoverse cores), 2n / wall time, best of 5"}


_CLOCK_C = r"""
#include <stdint.h>
uint64_t trioseq_clock_chain(uint64_t n, uint64_t x, uint64_t y) {
  for (uint64_t i = 0; i < n; i++) { x += y; y ^= x; }
  return x ^ y;
}
"""
_host_mhz = None


def measured_host_mhz():
    """Clock of the host core running the oracle, measured: gcc builds a loop whose iterations
    are one dependent integer add and xor (2 cycles at 1-cycle latency each; the loop counter
    runs beside them), and the clock is 2n cycles over the wall time. Used where the kernel
    exposes no frequency (no cpufreq, no CPPC nominal clock). None if gcc is missing."""
    global _host_mhz
    if _host_mhz is not None:
        return _host_mhz
    import ctypes
    import shutil
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        return None
    with tempfile.TemporaryDirectory() as d:
        src, lib = os.path.join(d, "clk.c"), os.path.join(d, "clk.so")
        with open(src, "w") as fh:
            fh.write(_CLOCK_C)
        if subprocess.run([cc, "-O2", "-shared", "-fPIC", src, "-o", lib],
                          capture_output=True).returncode != 0:
            return None
        fn = ctypes.CDLL(lib).trioseq_clock_chain
        fn.restype = ctypes.c_uint64
        fn.argtypes = [ctypes.c_uint64] * 3
        n, best = 100_000_000, 0.0
        for _ in range(5):
            t = time.perf_counter()
            fn(n, 1, 2)
            best = max(best, 2 * n / (time.perf_counter() - t) / 1e6)
    _host_mhz = round(best, 1)
    return _host_mhz


def cpu_all_cores_sample(triplets, sc, target_s: float = 3.0):
    """The oracle's batch entry on every host core (independent triplets, one per thread at a
    time), timed on a prefix of the batch sized for about target_s seconds."""
    import oracle
    n_cores = os.cpu_count() or 1
    probe = triplets[:8]
    t0 = time.perf_counter()
    oracle.align_many(probe, sc.sub, sc.gap)
    per_cell = (time.perf_counter() - t0) / sum(len(a) * len(b) * len(c) for a, b, c in probe)
    budget = target_s * n_cores / per_cell
    sample, tot = [], 0
    for t in triplets:
        sample.append(t)
        tot += len(t[0]) * len(t[1]) * len(t[2])
        if tot >= budget:
            break
    t0 = time.perf_counter()
    oracle.align_many(sample, sc.sub, sc.gap, threads=n_cores)
    dt = time.perf_counter() - t0
    return {"value": tot / dt / 1e9, "unit": "GCUPS", "cores": n_cores, "kind": "oracle",
            "sample": f"first {len(sample)} triplets of the batch ({tot} cells, {dt:.1f} s)",
            "host": host_cpu()}


def cpu_oracle_sample(w, target_cells: float, traceback: bool):
    """Time the oracle on prefixes of the workload's first triplet(s) (~target_cells cells)."""
    import oracle
    import numpy as np
    sc = w.scoring
    if len(w.triplets) == 1:
        t = w.triplets[0]
        L = int(round(target_cells ** (1.0 / 3.0)))
        L = max(8, min(L, min(len(x) for x in t)))
        sample = [tuple(np.ascontiguousarray(x[:L]) for x in t)]
        desc = f"prefixes of length {L} of the workload triplet"
    else:
        sample, tot = [], 0
        for t in w.triplets:
            sample.append(t)
            tot += len(t[0]) * len(t[1]) * len(t[2])
            if tot >= target_cells:
                break
        desc = f"first {len(sample)} triplets of the workload"
    cells = sum(len(a) * len(b) * len(c) for a, b, c in sample)
    t0 = time.perf_counter()
    for s in sample:
        oracle.align(*s, sc.sub, sc.gap, traceback=traceback)
    dt = time.perf_counter() - t0
    mode = "score + traceback" if traceback else "score only"
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"{desc} ({cells} cells, {mode}, {dt:.1f} s)", "host": host_cpu()}, dt


def run_reference(args, rank: int):
    if rank != 0:
        return
    ws = workloads()
    make, desc = ws[args.workload]
    w = make()
    tb = w.traceback
    import oracle
    oracle.build()
    # each step: a bounded sample (~2.5e7 cells) of the workload on one host core
    samples = []
    for i in range(args.warmup + args.steps):
        cb, dt = cpu_oracle_sample(w, 2.5e7, tb)
        if i >= args.warmup:
            samples.append((cb, dt))
    v = statistics.mean(c["value"] for c, _ in samples)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(dt for _, dt in samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": f"{w.name}: {desc}", "reference": "CPU oracle (C++, "
                       "int64), bounded prefix sample per step"},
            "cpu_baseline": dict(samples[-1][0], value=v),
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
def max_over_ranks(x: float, dist, device: str) -> float:
    """Slowest rank's value (every rank runs its own replica; no data-path collective)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_batch(B, torch, bt, steps: int, warmup: int, stream, flush, n):
    """Run a device-resident batch; returns (per-step event ms, per-step kernel ms, scores)."""
    B.trioseq_batch_profile(bt, True)
    for _ in range(warmup):
        B.trioseq_batch_run(bt, stream)
    torch.cuda.synchronize()
    step_ms, kern_ms, walk_ms = [], [], []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0.record(stream)
        B.trioseq_batch_run(bt, stream)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        k, wk = B.trioseq_batch_timing(bt)
        kern_ms.append(k)
        walk_ms.append(wk)
    scores = B.trioseq_batch_scores(bt, n, stream)
    return step_ms, kern_ms, walk_ms, scores


def _serve(B, srv, reqs, strs, rate, cap):
    """Submit `reqs` to the server with Poisson gaps at `rate` requests/s (None: all at once) and
    poll until every result is back. Returns submit times, completion times, results, tickets."""
    t_sub, t_done, tickets, results = {}, {}, [None] * len(reqs), {}
    fresh = []  # tickets submitted since the poller last took them (O(1) per poll pass)
    lock = threading.Lock()

    def submitter():
        t0 = time.perf_counter()
        at = 0.0
        for i, r in enumerate(reqs):
            if rate is not None:
                at += r["gap"] / rate
                while time.perf_counter() - t0 < at:
                    time.sleep(min(0.0005, max(0.0, at - (time.perf_counter() - t0))))
            mode = B.WITH_TRACEBACK if r["traceback"] else B.SCORE_ONLY
            while True:
                st, tk = B.trioseq_submit(srv, strs[i], 1 if r["protein"] else 0, mode)
                if st == B.OK:
                    break
                time.sleep(0.001)
            with lock:
                t_sub[tk] = time.perf_counter()
                tickets[i] = tk
                fresh.append(tk)

    th = threading.Thread(target=submitter)
    th.start()
    pending = set()
    n_done = 0
    while n_done < len(reqs):
        with lock:
            pending.update(fresh)
            fresh.clear()
        for tk in list(pending):
            st, score, rows = B.trioseq_poll(srv, tk, cap)
            if st == B.OK:
                t_done[tk] = time.perf_counter()
                results[tk] = (score, rows)
                pending.discard(tk)
                n_done += 1
        time.sleep(0.0002)
    th.join()
    return t_sub, t_done, results, tickets


def serving_golden(reqs, results):
    """Served results of the stream's first requests against the stored oracle values (scores,
    and the alignment digests of traceback requests): the number of requests checked, or None
    when no values are stored for these inputs. A mismatch stops the benchmark."""
    from tests.golden import goldens
    try:
        meta, want = goldens.load_config4()
    except (OSError, ValueError, AssertionError):
        return None
    n = len(want)
    if len(reqs) < n or meta.get("input_sha256") != goldens.input_digest(
            [r["triplet"] for r in reqs[:n]]):
        return None
    for wnt, (score, rows) in zip(want, results[:n]):
        assert score == wnt["score"], f"served request {wnt['id']}: score differs from the oracle"
        if wnt["traceback"]:
            assert goldens.rows_digest(rows) == wnt["rows_sha256"], \
                f"served request {wnt['id']}: alignment differs from the oracle"
    return {"requests_checked": n, "equal": True}


def cpu_all_cores_mix(reqs, dna, prot, target_s: float = 3.0):
    """The oracle on every host core over the serving mix, replayed in arrival order: a prefix of
    the requests sized for about target_s seconds, each scoring scheme's requests as one
    multi-threaded batch (scores only; the oracle has no batched traceback)."""
    import oracle
    n_cores = os.cpu_count() or 1
    vol = [len(r["triplet"][0]) * len(r["triplet"][1]) * len(r["triplet"][2]) for r in reqs]
    probe = [r["triplet"] for r in reqs[:8] if not r["protein"]][:4]
    t0 = time.perf_counter()
    oracle.align_many(probe, dna.sub, dna.gap)
    per_cell = (time.perf_counter() - t0) / max(1, sum(
        len(a) * len(b) * len(c) for a, b, c in probe))
    budget = target_s * n_cores / per_cell
    n, tot = 0, 0
    while n < len(reqs) and tot < budget:
        tot += vol[n]
        n += 1
    groups = [[r["triplet"] for r in reqs[:n] if r["protein"] == p] for p in (False, True)]
    t0 = time.perf_counter()
    for trips, sc in zip(groups, (dna, prot)):
        if trips:
            oracle.align_many(trips, sc.sub, sc.gap, threads=n_cores)
    dt = time.perf_counter() - t0
    return {"value": tot / dt / 1e9, "unit": "GCUPS", "cores": n_cores, "kind": "oracle",
            "sample": f"first {n} requests of the mix in arrival order ({len(groups[0])} DNA, "
                      f"{len(groups[1])} protein; {tot} cells, scores only, {dt:.1f} s)",
            "host": host_cpu()}


def serving_measurement(B, n_req: int = 10000, load: float = 0.7, n_cal: int = 1000,
                        cpu_legs: bool = True):
    """Serving stream: mixed DNA/protein requests (20% traceback). The server's capacity on this
    mix is measured first with closed-loop bursts (n_cal requests spread evenly over the stream,
    submitted at once; the lower of two bursts); the stream
    then arrives with Poisson gaps at `load` x that capacity. Latency = submit to the poll that
    returns the result. A few served results are re-aligned alone and must match exactly."""
    from paper_2605_28400_gb300 import synth
    dna, prot, reqs = synth.config4(n=n_req)
    plans = [B.trioseq_plan(dna.alphabet, dna.sub, dna.gap),
             B.trioseq_plan(prot.alphabet, prot.sub, prot.gap)]
    cells = [len(r["triplet"][0]) * len(r["triplet"][1]) * len(r["triplet"][2]) for r in reqs]
    mean_cells = sum(cells) / len(cells)
    strs = [[synth.to_str(s, (prot if r["protein"] else dna).alphabet) for s in r["triplet"]]
            for r in reqs]
    cap = 3 * max(len(s) for st in strs for s in st) + 16
    # capacity: a burst of n_cal requests taken evenly across the whole stream, so that its mix is
    # the stream's (the first n_cal alone drew capacities 5-10% apart between runs, and the offered
    # load with them: p99 27-109 ms at a nominal 70%)
    cal = list(range(0, len(reqs), max(1, len(reqs) // n_cal)))[:n_cal]
    cal_cells = sum(cells[i] for i in cal)
    bursts = []
    for _ in range(2):  # the lower of two bursts
        srv = B.trioseq_server_create(plans)
        ts, td, _, _ = _serve(B, srv, [reqs[i] for i in cal], [strs[i] for i in cal], None, cap)
        B.trioseq_server_destroy(srv)
        bursts.append(cal_cells / (max(td.values()) - min(ts.values())) / 1e9)
    capacity = min(bursts)
    # The same n_cal requests as four plain batches, one per (scheme, mode) group, back to back
    # (host strings in, results out, one trioseq_align_batch each): what the server's burst is
    # compared with, so that the gap splits into the mix's own cost and serving's overhead.
    groups = {}
    for i in cal:
        groups.setdefault((reqs[i]["protein"], reqs[i]["traceback"]), []).append(i)
    batched_mix = 0.0
    for rep in range(3):  # the first pass sizes the plans' workspaces; the best of the next two
        t0 = time.perf_counter()
        for (prot_, tb_), idx in groups.items():
            B.trioseq_align_batch(plans[1 if prot_ else 0], [strs[i] for i in idx],
                                  B.WITH_TRACEBACK if tb_ else B.SCORE_ONLY)
        if rep > 0:
            batched_mix = max(batched_mix, cal_cells / (time.perf_counter() - t0) / 1e9)
    rate = load * capacity * 1e9 / mean_cells  # requests per second
    srv = B.trioseq_server_create(plans)
    t_sub, t_done, results, tickets = _serve(B, srv, reqs, strs, rate, cap)
    B.trioseq_server_destroy(srv)
    lat = sorted(1e3 * (t_done[tk] - t_sub[tk]) for tk in t_done)
    span = max(t_done.values()) - min(t_sub.values())
    same = True
    for i in (0, 1, 2, len(reqs) // 2, len(reqs) - 1):
        r = reqs[i]
        mode = B.WITH_TRACEBACK if r["traceback"] else B.SCORE_ONLY
        pl = plans[1 if r["protein"] else 0]
        alone = B.trioseq_align_batch(pl, [strs[i]], mode)
        score, rows = results[tickets[i]]
        same &= score == int(alone[0])
        if r["traceback"]:
            same &= rows == B.trioseq_traceback(pl, 0)
    for p in plans:
        B.trioseq_plan_destroy(p)
    golden = serving_golden(reqs, [results[tickets[i]] for i in range(len(reqs))])
    return {"requests": len(reqs), "arrival_rate_per_s": rate,
            "equals_oracle_on_stored_prefix": golden,
            "server_capacity_gcups": capacity, "capacity_burst_requests": len(cal),
            "capacity_bursts_gcups": bursts,
            "same_mix_as_four_batches_gcups": batched_mix,
            "load_vs_server_capacity": load,
            "mean_cells_per_request": mean_cells, "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "max_ms": lat[-1],
            "aggregate_gcups": sum(cells) / span / 1e9, "span_s": span,
            "identical_to_alone_sample": bool(same),
            "cpu_all_cores": cpu_all_cores_mix(reqs, dna, prot) if cpu_legs else None,
            "mix": "70% DNA / 30% protein, 20% traceback, ancestor lognormal(ln 300, 0.8) "
                   "clipped to [50, 2000]"}


def aux_measurements(B, torch, stream, flush, sms, clock_mhz, skip: str, cpu_legs: bool = True,
                     lanes: float = INT32_LANES_PER_SM):
    """Secondary lines of the metric: the traceback workload (related DNA triplet n~1000, score +
    4-bit codes + walk), the semi-global and local types on the n=4000 protein triplet, the
    4096-triplet batch in one persistent launch versus one launch per triplet, and the serving
    stream (p50/p99 latency)."""
    from paper_2605_28400_gb300 import synth
    out = {}
    for key in ("dna1000", "protein4000", "dna128"):
        if key == skip:
            continue
        make, desc = workloads()[key]
        w = make()
        plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
        mode = B.WITH_TRACEBACK if w.traceback else B.SCORE_ONLY
        tuned = B.trioseq_plan_autotune(plan, triplet_strings(w), mode)
        bt = B.trioseq_batch_create(plan, triplet_strings(w), mode)
        sm, km, wk, sc = time_batch(B, torch, bt, 10, 3, stream, flush, 1)
        binfo = B.trioseq_batch_info(bt)
        tile, kname = kernel_of(binfo, len(w.triplets))
        packing = binfo.get("packing", 1)
        kmean = statistics.mean(km)
        ach = OPS_PER_CELL * w.cells / (kmean / 1e3) / 1e12
        peak = packing * sms * lanes * clock_mhz * 1e6 / 1e12
        entry = {"workload": f"{w.name}: {desc}",
                 "gcups": w.cells / (statistics.mean(sm) / 1e3) / 1e9,
                 "ms_per_step": statistics.mean(sm), "kernel_ms": kmean, "cells": w.cells,
                 "score": int(sc[0]), "tuned": tuned,
                 "tile": tile,
                 "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                              "unit": "TOPS (int32)" if packing == 1 else "TOPS (int16x2 lanes)",
                              "frac": ach / peak, "kernel": kname,
                              "traffic": measured_traffic(key, tile)}}
        if w.traceback:
            entry["walk_ms"] = statistics.mean(wk)
            entry["roofline"]["code_stream_gbs"] = CODE_BYTES_PER_CELL * w.cells / kmean / 1e6
        entry["equals_oracle"] = check_golden(
            key, w, sc, B.trioseq_batch_alignment(bt, 0) if w.traceback else None)
        out[key] = entry
        B.trioseq_batch_destroy(bt)
        B.trioseq_plan_destroy(plan)

    # The n=4000 protein triplet on the int32 8x8 kernel (one cell per register lane), the
    # kernel the two-cells-per-register one is measured against; interval 16, its best there.
    w = synth.config3()
    os.environ["TRIOSEQ_SCORE_TILE"], os.environ["TRIOSEQ_TI"] = "8x8", "16"
    try:
        plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    finally:
        os.environ.pop("TRIOSEQ_SCORE_TILE", None)
        os.environ.pop("TRIOSEQ_TI", None)
    bt = B.trioseq_batch_create(plan, triplet_strings(w), B.SCORE_ONLY)
    binfo = B.trioseq_batch_info(bt)
    assert binfo["packing"] == 1 and binfo["tile"] == (8, 8)
    sm, km, _, sc = time_batch(B, torch, bt, 5, 3, stream, flush, 1)
    kmean = statistics.mean(km)
    ach = OPS_PER_CELL * w.cells / (kmean / 1e3) / 1e12
    peak = sms * lanes * clock_mhz * 1e6 / 1e12
    out["protein4000_int32_8x8"] = {
        "workload": f"{w.name}: the main line's triplet on the int32 kernel (tile 8x8, interval 16)",
        "gcups": w.cells / (statistics.mean(sm) / 1e3) / 1e9, "kernel_ms": kmean,
        "score": int(sc[0]), "dtype": "int32", "equals_oracle": check_golden("protein4000", w, sc),
        "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TOPS (int32)",
                     "frac": ach / peak, "kernel": "wavefront_kernel<8,8>",
                     "traffic": measured_traffic("protein4000", "8x8")}}
    B.trioseq_batch_destroy(bt)
    B.trioseq_plan_destroy(plan)

    # Semi-global and local types (Sec. II) on the n=4000 protein triplet, score only. Both are
    # counted at the metric's 13 algorithmic int32 ops per cell. Local also does the v = 0
    # candidate and the running best per cell (15 ops): its fraction at 15 is reported beside.
    w = synth.config3()
    for flags, name, extra in ((B.SEMIGLOBAL, "semiglobal", 0), (B.LOCAL, "local", 2)):
        ops = OPS_PER_CELL
        plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap, flags)
        tuned = B.trioseq_plan_autotune(plan, triplet_strings(w), B.SCORE_ONLY)
        bt = B.trioseq_batch_create(plan, triplet_strings(w), B.SCORE_ONLY)
        binfo = B.trioseq_batch_info(bt)
        packing = binfo.get("packing", 1)
        sm, km, _, sc = time_batch(B, torch, bt, 5, 3, stream, flush, 1)
        kmean = statistics.mean(km)
        ach = ops * w.cells / (kmean / 1e3) / 1e12
        peak = packing * sms * lanes * clock_mhz * 1e6 / 1e12
        out[f"protein4000_{name}"] = {
            "workload": f"{w.name}: alignment type {name} (Sec. II), score only",
            "gcups": w.cells / (statistics.mean(sm) / 1e3) / 1e9, "kernel_ms": kmean,
            "score": int(sc[0]), "tuned": tuned, "ops_per_cell": ops,
            "tile": binfo["tile_label"], "kernel": binfo["kernel"],
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak,
                         "unit": "TOPS (int32)" if packing == 1 else "TOPS (int16x2 lanes)",
                         "frac": ach / peak}}
        if extra:
            out[f"protein4000_{name}"]["roofline"]["frac_counting_type_ops"] = {
                "ops_per_cell": ops + extra, "frac": (ops + extra) / ops * ach / peak}
        B.trioseq_batch_destroy(bt)
        B.trioseq_plan_destroy(plan)

    w = synth.config2()
    strs = triplet_strings(w)
    plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    tuned_batch = B.trioseq_plan_autotune(plan, strs, B.SCORE_ONLY)
    bt = B.trioseq_batch_create(plan, strs, B.SCORE_ONLY)
    packing = B.trioseq_batch_info(bt)["packing"]
    sm, km, _, sc_batched = time_batch(B, torch, bt, 5, 2, stream, flush, len(strs))
    batched = w.cells / (statistics.mean(sm) / 1e3) / 1e9
    kb = statistics.mean(km)
    ach_b = OPS_PER_CELL * w.cells / (kb / 1e3) / 1e12
    peak_b = packing * sms * lanes * clock_mhz * 1e6 / 1e12
    B.trioseq_batch_destroy(bt)
    singles = [B.trioseq_batch_create(plan, [s], B.SCORE_ONLY) for s in strs]
    for b in singles:  # untimed first run of each (captures its graph)
        B.trioseq_batch_run(b, stream)
    torch.cuda.synchronize()
    reps = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(2):
        if flush is not None:
            flush.zero_()
        e0.record(stream)
        for b in singles:
            B.trioseq_batch_run(b, stream)
        e1.record(stream)
        e1.synchronize()
        reps.append(e0.elapsed_time(e1))
    same = all(int(B.trioseq_batch_scores(b, 1, stream)[0]) == int(sc_batched[i])
               for i, b in enumerate(singles))
    for b in singles:
        B.trioseq_batch_destroy(b)
    B.trioseq_plan_destroy(plan)
    per_triplet = w.cells / (statistics.mean(reps) / 1e3) / 1e9
    out["batch4096_score_only"] = {
        "equals_oracle": check_golden("batch4096", w, sc_batched),
        "batched_gcups": batched, "per_triplet_launch_gcups": per_triplet,
        "batched_over_per_triplet": batched / per_triplet, "identical_scores": bool(same),
        "tuned_batched": tuned_batch, "packing": packing, "kernel_ms": kb,
        "cpu_all_cores": cpu_all_cores_sample(w.triplets, w.scoring) if cpu_legs else None,
        "roofline": {"bound": "alu", "achieved": ach_b, "peak": peak_b,
                     "unit": "TOPS (int32)" if packing == 1 else "TOPS (int16x2 lanes)",
                     "frac": ach_b / peak_b},
        "cells": w.cells}
    # The same 4096 triplets with traceback: the traceback kernels and the walk at full occupancy
    # (thousands of independent triplets), where the single-triplet line is bound by its ramp.
    plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    tuned_tb = B.trioseq_plan_autotune(plan, strs, B.WITH_TRACEBACK)
    bt = B.trioseq_batch_create(plan, strs, B.WITH_TRACEBACK)
    sm, km, wk, sc_tb = time_batch(B, torch, bt, 3, 2, stream, flush, len(strs))
    B.trioseq_batch_destroy(bt)
    B.trioseq_plan_destroy(plan)
    kt = statistics.mean(km)
    ach_t = OPS_PER_CELL * w.cells / (kt / 1e3) / 1e12
    peak_t = sms * lanes * clock_mhz * 1e6 / 1e12
    out["batch4096_traceback"] = {
        "workload": "the 4096-triplet batch with 4-bit traceback codes and one walk per triplet",
        "gcups": w.cells / (statistics.mean(sm) / 1e3) / 1e9, "ms_per_step": statistics.mean(sm),
        "kernel_ms": kt, "walk_ms": statistics.mean(wk), "tuned": tuned_tb,
        "identical_scores_to_score_only": [int(x) for x in sc_tb] == [int(x) for x in sc_batched],
        "roofline": {"bound": "alu", "achieved": ach_t, "peak": peak_t, "unit": "TOPS (int32)",
                     "frac": ach_t / peak_t,
                     "code_stream_gbs": CODE_BYTES_PER_CELL * w.cells / kt / 1e6},
        "cells": w.cells}
    out["batch4096_affine"] = affine_measurement(B, torch, stream, flush, sms, clock_mhz, lanes)
    out["serving_stream"] = serving_measurement(B, cpu_legs=cpu_legs)
    out["dna8000_linear_space_traceback"] = linear_space_measurement(B, torch, stream)
    return out


# Affine gaps (natural gap costs): algorithmic int32 work per cell. Each of the 13 reachable
# states takes the best of its (move, previous state) candidates: 4 moves with two or three
# residues x 13 states plus 3 single-residue moves x 13 = 91 candidates, an add and a max each.
AFFINE_OPS_PER_CELL = 2 * 91


def affine_measurement(B, torch, stream, flush, sms, clock_mhz, lanes):
    """The 4096-triplet DNA batch under affine gaps (trioseq_plan_affine: alpha = -2 per residue
    against a gap, gamma = -4 per maximal gap run of a pair), score only, one persistent launch.
    The first 64 scores are checked against the stored oracle values."""
    from paper_2605_28400_gb300 import synth
    from tests.golden import goldens
    w = synth.config2()
    strs = triplet_strings(w)
    plan = B.trioseq_plan_affine(w.scoring.alphabet, w.scoring.sub, w.scoring.gap,
                                 goldens.AFFINE_GAP_OPEN)
    try:
        bt = B.trioseq_batch_create(plan, strs, B.SCORE_ONLY)
        sm, km, _, sc = time_batch(B, torch, bt, 3, 1, stream, flush, len(strs))
        B.trioseq_batch_destroy(bt)
    finally:
        B.trioseq_plan_destroy(plan)
    checked = None
    try:
        meta, want = goldens.load_config2_affine()
        if meta.get("input_sha256") == goldens.input_digest(w.triplets[:len(want)]):
            assert [int(x) for x in sc[:len(want)]] == [int(x) for x in want], \
                "affine batch: scores differ from the stored oracle values"
            checked = len(want)
    except OSError:
        pass
    kmean = statistics.mean(km)
    ach = AFFINE_OPS_PER_CELL * w.cells / (kmean / 1e3) / 1e12
    peak = sms * lanes * clock_mhz * 1e6 / 1e12
    return {"workload": f"{w.name}: affine gaps (natural gap costs, alpha -2, gamma "
                        f"{goldens.AFFINE_GAP_OPEN}), score only",
            "gcups": w.cells / (statistics.mean(sm) / 1e3) / 1e9, "kernel_ms": kmean,
            "cells": w.cells, "equals_oracle_first": checked, "kernel": "affine_kernel",
            "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TOPS (int32)",
                         "frac": ach / peak, "ops_per_cell": AFFINE_OPS_PER_CELL}}


def linear_space_measurement(B, torch, stream):
    """Score + traceback of one related DNA triplet at ancestor length 8000 (5.1e11 cells). Its
    4-bit code cube alone would take ~256 GB, so the batch runs in slabs: a forward pass keeps a
    plane per slab boundary, then each slab is recomputed with codes from the top down while the
    walk continues through it. Checks: the score equals the score-only run, and the aligned rows
    with gaps removed are the inputs."""
    make, desc = workloads()["dna8000"]
    w = make()
    strs = triplet_strings(w)
    plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    try:
        bt = B.trioseq_batch_create(plan, strs, B.WITH_TRACEBACK)
        info = B.trioseq_batch_info(bt)
        B.trioseq_batch_run(bt, stream)
        B.trioseq_batch_scores(bt, 1, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = []
        for _ in range(2):
            e0.record(stream)
            B.trioseq_batch_run(bt, stream)
            e1.record(stream)
            e1.synchronize()
            reps.append(e0.elapsed_time(e1))
        score = int(B.trioseq_batch_scores(bt, 1, stream)[0])
        rows = B.trioseq_batch_alignment(bt, 0)
        B.trioseq_batch_destroy(bt)
        score_only = int(B.trioseq_align_batch(plan, strs, B.SCORE_ONLY, stream)[0])
    finally:
        B.trioseq_plan_destroy(plan)
    ms = statistics.mean(reps)
    return {"workload": f"{w.name}: {desc}", "cells": w.cells,
            "gcups": w.cells / (ms / 1e3) / 1e9, "ms": ms,
            "slab_slices": info["slab_slices"], "slabs": info["slabs"],
            "code_cube_gb_if_stored_whole": w.cells * CODE_BYTES_PER_CELL / 1e9,
            "alignment_columns": len(rows[0]), "score": score,
            "score_equals_score_only_run": score == score_only,
            "rows_strip_to_inputs": all(r.replace("-", "") == s for r, s in zip(rows, strs[0]))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(workloads()), default="protein4000")
    ap.add_argument("--no-aux", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--tile", default=None,
                    help="force the wavefront tile (e.g. 8x16, 8x8v, 8x8, 8x4) instead of autotuning")
    ap.add_argument("--ti", type=int, default=None,
                    help="progress interval with --tile (default: the plan's, 8)")
    ap.add_argument("--alu-rate", action="store_true",
                    help="print the measured int32 instruction-form rates (trioseq_alu_rate) and exit")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.alu_rate:  # the roofline's denominator alone (one GPU, no workload)
        from paper_2605_28400_gb300 import binding as B
        print(json.dumps(measured_alu(B)))
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2605_28400_gb300 import binding as B
    B.load()
    make, desc = workloads()[args.workload]
    wg, gdesc = global_workload(args.workload, world) if world > 1 else (None, None)
    if wg is not None:  # a batch: shard its triplets over the ranks (Sec. V-D)
        desc = gdesc
        w, rank_cells = shard_workload(wg, world, rank, B)
        cells_total = wg.cells
        parallelism = (f"dp{world}: triplets sharded by the dynamic partition (Sec. V-D), "
                       "largest first")
    else:  # one triplet, or one GPU: every rank aligns its own replica
        w = make()
        rank_cells = [w.cells] * world
        cells_total = world * w.cells
        parallelism = f"dp{world}: replicas" if world > 1 else "single GPU"
    tb = w.traceback
    mode = B.WITH_TRACEBACK if tb else B.SCORE_ONLY
    strs = triplet_strings(w)
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    uuid = str(getattr(props, "uuid", "") or "")
    uuid = uuid if uuid.startswith("GPU-") else (f"GPU-{uuid}" if uuid else None)

    if args.tile:  # a forced tile (profiling one kernel): no autotuner launches before it
        os.environ["TRIOSEQ_TB_TILE" if tb else "TRIOSEQ_SCORE_TILE"] = args.tile
        if args.ti:
            os.environ["TRIOSEQ_TI"] = str(args.ti)
    plan = B.trioseq_plan(w.scoring.alphabet, w.scoring.sub, w.scoring.gap)
    for k in ("TRIOSEQ_TB_TILE", "TRIOSEQ_SCORE_TILE", "TRIOSEQ_TI"):
        if args.tile:
            os.environ.pop(k, None)
    if args.tile:
        tuned = {"tile": None, "ti": args.ti or 8, "forced": args.tile}
    else:
        tuned = B.trioseq_plan_autotune(plan, strs, mode)  # untimed: picks tile and interval
    bt = B.trioseq_batch_create(plan, strs, mode)
    info = B.trioseq_batch_info(bt)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    sampler = ClockSampler(uuid)
    time.sleep(0.2)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    step_ms, kern_ms, walk_ms, scores = time_batch(B, torch, bt, args.steps, args.warmup, stream,
                                                   flush, len(strs))
    torch.cuda.synchronize()
    t1 = time.time()
    if dist:
        dist.barrier()
    clocks = sampler.summary(t0, t1)

    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    ms_step = total_ms / args.steps
    value = cells_total / (ms_step / 1e3) / 1e9

    # e2e through the public C call on host strings
    e2e_ms = []
    for i in range(max(3, min(args.steps, 20)) + 2):
        torch.cuda.synchronize()
        a = time.perf_counter()
        s2 = B.trioseq_align_batch(plan, strs, mode, stream)
        if tb:
            B.trioseq_traceback(plan, 0)
        e2e_ms.append((time.perf_counter() - a) * 1e3)
    e2e_ms = e2e_ms[2:]
    h2d, d2h = B.trioseq_plan_io_bytes(plan)
    assert s2.tolist() == scores.tolist(), "e2e and device-resident scores differ"
    e2e_total = max_over_ranks(sum(e2e_ms), dist, "cuda")
    e2e_val = cells_total / (e2e_total / len(e2e_ms) / 1e3) / 1e9

    clock_mhz = clocks.get("sm_mhz") or 2070.0
    try:
        alu = measured_alu(B)
    except Exception as exc:  # the nominal lane count stands; the line says why
        alu = {"error": str(exc)}
    lanes = roof_lanes(alu if "int32_ops_per_clk_per_sm" in alu else None)
    kmean = statistics.mean(kern_ms)
    achieved = OPS_PER_CELL * w.cells / (kmean / 1e3) / 1e12
    # packed int16x2 batches run two cells per instruction lane: the lane roof doubles
    packing = info.get("packing", 1)
    tile, kname = kernel_of(info, len(strs))
    peak = packing * sms * lanes * clock_mhz * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TOPS (int32)" if packing == 1 else "TOPS (int16x2 lanes)",
            "frac": achieved / peak,
            "traffic": measured_traffic(args.workload, tile),
            "kernel": kname, "kernel_ms": kmean,
            "peak_basis": f"{sms} SMs x {lanes:.1f} int32 ops/clk (the lower of the nominal "
                          f"{INT32_LANES_PER_SM} and the measured rate) x median SM clock "
                          f"{clock_mhz:.0f} MHz sampled in the timed region"
                          + (" x 2 (int16x2 packing)" if packing == 2 else ""),
            "alu_measured": alu}
    if packing == 2:  # the metric's int32 roof, beside the roof of the int16x2 lanes used
        roof["frac_of_int32_roof"] = achieved / (peak / 2)
    if tb:
        roof["code_stream_gbs"] = CODE_BYTES_PER_CELL * w.cells / (kmean / 1e3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("int32" if packing == 1 else
                      "int16x2 (two cells per 32-bit register, each a 16-bit value relative to "
                      "a per-task base; exact by the range bound, boundary records int32)"
                      if len(strs) == 1 else
                      "int16x2 (two triplets per 32-bit register; exact by the range bound)"),
            "data": "synthetic",
            "config": {"workload": f"{(wg or w).name}: {desc}", "cells_per_step": cells_total,
                       "cells_per_rank": rank_cells,
                       "triplets": len(wg.triplets) if wg else world * len(strs),
                       "mode": "score+traceback" if tb else "score",
                       "column_tasks": info["tasks"],
                       "tile": tile,
                       "progress_interval": tuned["ti"], "autotuned": not args.tile,
                       "l2": "256 MiB flush between timed steps (outside the events)",
                       "parallelism": parallelism},
            "roofline": roof,
            "e2e": {"value": e2e_val, "unit": "GCUPS", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h), "ms_per_step": statistics.mean(e2e_ms)},
            "gpu_launches": world * args.steps * (2 if tb else 1),
            "clocks": clocks,
            "score": int(scores[0]),
            "equals_oracle": check_golden(args.workload, w, scores,
                                          B.trioseq_batch_alignment(bt, 0) if tb and
                                          len(strs) == 1 else None) if wg is None else None}
    B.trioseq_batch_destroy(bt)
    B.trioseq_plan_destroy(plan)

    # aux lines and the CPU baseline: one GPU only (at N > 1 the other GPUs would idle meanwhile)
    if rank == 0 and world == 1 and not args.no_aux:
        line["aux"] = aux_measurements(B, torch, stream, flush, sms, clock_mhz, args.workload,
                                       not args.no_cpu, lanes)
    if rank == 0 and world == 1 and not args.no_cpu:
        cb, _ = cpu_oracle_sample(w, 1e9, tb)  # ~15 s of one host core
        line["cpu_baseline"] = cb
    sampler.stop()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
