"""The N>1 path of the benchmark on CPU: two gloo ranks, each an independent
replica (no data-path collective). The whole-job value is the units of all
ranks over the slowest rank's time, and only rank 0 runs the oracle arm."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import bench

    ranks = bench.Ranks()
    try:
        # rank r processed (r+1)*100 units in (r+1)*2 seconds
        units, sec = (rank + 1) * 100.0, (rank + 1) * 2.0
        got = {"max": ranks.max(sec), "sum": ranks.sum(units), "rate": ranks.rate(units, sec)}
        args = bench.parse_args(["--impl", "reference", "--gpus", str(world)])
        if rank != 0:
            got["reference_rc"] = bench.run_reference(args, ranks)
        ranks.barrier()
        q.put((rank, got))
    finally:
        ranks.close()


def test_two_gloo_ranks_aggregate_as_replicas():
    pytest.importorskip("torch.distributed")
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r]["max"] == 4.0 and out[r]["sum"] == 300.0
        assert out[r]["rate"] == pytest.approx(300.0 / 4.0)
    # the oracle arm runs on rank 0 only; the other ranks return at once
    assert out[1]["reference_rc"] == 0


def test_reference_arm_line_on_cpu(capsys):
    """The reference arm (the oracle) prints the benchmark's JSON line with
    the keys the contract asks for; run here on the small uniform workload."""
    import json

    import bench

    rc = bench.main(["--impl", "reference", "--workload", "uniform-3d-100k", "--steps", "1", "--warmup", "0"])
    assert rc == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == "uniform-3d-100k"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
