"""Multi-rank logic of the benchmark, on CPU with gloo (world size 2).

The path shards over independent triplets with no collective on the data path: a batch is split
over the ranks by the dynamic partition of Sec. V-D, a single triplet runs as one replica per
rank, and the only cross-rank step is taking the slowest rank's time. The reference arm runs on
rank 0 only and the other ranks exit cleanly without output.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(values[rank], dist, "cpu")
        out_q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    values = [3.5, 7.25]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, values, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 7.25, 1: 7.25}


def test_max_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_prints_contract_line():
    import json

    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GCUPS" and line["value"] > 0
    assert line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_roofline_lanes_take_the_lower_of_nominal_and_measured():
    import bench
    assert bench.roof_lanes(None) == bench.INT32_LANES_PER_SM
    assert bench.roof_lanes({"int32_ops_per_clk_per_sm": 127.2}) == 127.2
    assert bench.roof_lanes({"int32_ops_per_clk_per_sm": 140.0}) == bench.INT32_LANES_PER_SM


def test_kernel_label_and_tile_checked_traffic(tmp_path, monkeypatch):
    import json

    import bench
    # the tile label and kernel come from the library's own report (trioseq_batch_kernel)
    assert bench.kernel_of({"tile": (8, 16), "packing": 2, "tile_label": "8x16s",
                            "kernel": "wavefront_vl_kernel<8,8,1>"}, 1) == \
        ("8x16s", "wavefront_vl_kernel<8,8,1>")
    # which sources a tile's traffic figure is tied to
    assert bench.kernel_source_hash("8x8v") == bench.kernel_source_hash("8x16s")
    assert bench.kernel_source_hash("8x8v") == bench.kernel_source_hash("8x16t")
    assert bench.kernel_source_hash("8x8v") == bench.kernel_source_hash("8x16")
    assert bench.kernel_source_hash("8x8v") != bench.kernel_source_hash("8x4")
    # traffic is reported only for the measured tile and the current kernel source
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "wavefront_traffic.json").write_text(json.dumps({"w": {
        "kernel_hash": "h0", "tile": "8x8v", "dram_bytes_per_launch": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda tile: "h0")
    assert bench.measured_traffic("w", "8x8v") == 123
    assert bench.measured_traffic("w", "8x16v") is None
    assert bench.measured_traffic("other", "8x8v") is None
    # a per-tile entry ("key/tile") where a workload's tiles are measured separately
    (prof / "wavefront_traffic.json").write_text(json.dumps({
        "w/8x8v": {"kernel_hash": "h0", "tile": "8x8v", "dram_bytes_per_launch": 5},
        "w/8x16": {"kernel_hash": "h0", "tile": "8x16", "dram_bytes_per_launch": 7}}))
    assert bench.measured_traffic("w", "8x8v") == 5
    assert bench.measured_traffic("w", "8x16") == 7
    assert bench.measured_traffic("w", "8x8") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda tile: "h1")  # source changed since
    assert bench.measured_traffic("w", "8x8v") is None


def _shard_worker(rank, world, port, out_q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2605_28400_gb300 import binding as B
    from paper_2605_28400_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.config2(seed=77, n=24, lo=4, hi=30)
        share, cells = bench.shard_workload(w, world, rank, B)
        scores = oracle.align_many(share.triplets, w.scoring.sub, w.scoring.gap).tolist()
        mine = [[int(len(s)) for s in t] + [sc] for t, sc in zip(share.triplets, scores)]
        gathered = [None] * world  # the test's own check; the bench has no collective
        dist.all_gather_object(gathered, (mine, share.cells, cells))
        out_q.put((rank, gathered))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_gloo_world2():
    """Two CPU ranks shard a batch by the dynamic partition (bench.shard_workload), each aligns
    its share with the oracle: every triplet is aligned exactly once, the union of the shares'
    results equals the whole batch aligned in one process, and every rank agrees on the loads."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    import oracle
    from paper_2605_28400_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got[0] == got[1]
    shares = got[0]
    w = synth.config2(seed=77, n=24, lo=4, hi=30)
    whole = oracle.align_many(w.triplets, w.scoring.sub, w.scoring.gap).tolist()
    want = sorted([int(len(s)) for s in t] + [sc] for t, sc in zip(w.triplets, whole))
    assert sorted(row for mine, _, _ in shares for row in mine) == want
    assert [c for _, c, _ in shares] == shares[0][2]  # each share's cells = its rank's load
    assert sum(shares[0][2]) == w.cells
    assert all(len(mine) > 0 for mine, _, _ in shares)


def test_all_core_oracle_replay_of_the_serving_mix():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_28400_gb300 import synth

    dna, prot, reqs = synth.config4(n=40, hi=120)
    got = bench.cpu_all_cores_mix(reqs, dna, prot, target_s=0.05)
    assert got["kind"] == "oracle" and got["value"] > 0 and got["cores"] >= 1
    assert "requests of the mix" in got["sample"]


def test_global_batch_extends_the_single_gpu_batch():
    """At N ranks the batch workload is N x 4096 triplets of the same recipe and seed; the
    generator is counter-based per triplet, so the first 4096 are the single-GPU batch."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    from paper_2605_28400_gb300 import synth

    wg, desc = bench.global_workload("batch4096", 2)
    one = synth.config2()
    assert len(wg.triplets) == 8192 and desc.startswith("8192 related DNA triplets")
    for t in (0, 1, 2047, 4095):
        assert all(np.array_equal(x, y) for x, y in zip(wg.triplets[t], one.triplets[t]))
    assert bench.global_workload("protein4000", 2) == (None, None)
