"""The benchmark's multi-rank path on CPU: two gloo ranks, each timing its own
subcarrier shard; the job time is the maximum over ranks and the aggregate
throughput counts every rank's bits (weak scaling, no data-path exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_env()
        assert (w, r, l) == (world, rank, rank)
        bench.barrier(world)
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        job_ms = bench.max_over_ranks(local_ms, world)
        q.put((rank, job_ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_reference_arm_only_rank0_prints(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1"])) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(capsys, monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys: the oracle timed on host cores, its own e2e object with no copies."""
    import json
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    assert bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "3"])) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["value"] > 0
    assert d["warmup"] >= 3 and d["higher_is_better"] is True and "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_oracle_rows_beside_the_gpu_rows():
    """cpu_baseline.rows: the oracle timed on a sample of every other measured
    row (downlink, BOX / BPSK prox, U = 32, soft outputs), scaled to a frame."""
    import bench
    rows = bench.cpu_rows(0.05)
    assert set(rows) == {"downlink", "box_prox", "bpsk_prox", "soft_outputs", "mixed_u32", "soft_outputs_u32"}
    for name, r in rows.items():
        assert r["ms_per_frame"] > 0 and r["gbit_s"] > 0 and " of " in r["sample"], name
