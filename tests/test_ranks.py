"""The N>1 paths on CPU with two gloo ranks: the benchmark's replicas (no
data-path collective; the whole-job value is the units of all ranks over the
slowest rank's time, and only rank 0 runs the oracle arm), and the
partitioned MTTKRP (each rank the partial result over its part of the store,
then one all-reduce), with the oracle standing in for the GPU kernel."""

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


def _shard_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2201_12523_gb300 import blco

    dist.init_process_group("gloo")
    try:
        rng = np.random.default_rng(5)
        dims = (40, 30, 20, 10)
        c = np.unique(np.stack([rng.integers(0, d, 3000) for d in dims], 1), axis=0)
        rng.shuffle(c)
        v = rng.random(len(c))
        A = [rng.standard_normal((d, 8)) for d in dims]
        st = oracle.build_store(c, v.astype(np.float32), dims, 64, 1 << 27)  # the store order
        cs = c[st.perm]
        vs = v[st.perm]
        got = []
        for mode in range(4):
            def part(begin, end, out, mode=mode):
                M, _ = oracle.mttkrp(cs[begin:end], vs[begin:end], dims, A, mode)
                out.copy_(torch.from_numpy(M))
            out = torch.zeros((dims[mode], 8), dtype=torch.float64)
            blco.sharded_sum(len(c), part, out)
            got.append(out.numpy())
        q.put((rank, got, len(c)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_partitioned_mttkrp_sums_to_the_full_result(world):
    """Each rank computes the MTTKRP of its part of the store order (the
    oracle in place of the kernel) and one all-reduce sums the parts: every
    rank must hold the oracle's MTTKRP of the whole tensor, for every mode."""
    pytest.importorskip("torch.distributed")
    import numpy as np

    import oracle

    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict((r, (g, n)) for r, g, n in (q.get(timeout=180) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(5)
    dims = (40, 30, 20, 10)
    c = np.unique(np.stack([rng.integers(0, d, 3000) for d in dims], 1), axis=0)
    rng.shuffle(c)
    v = rng.random(len(c))
    A = [rng.standard_normal((d, 8)) for d in dims]
    for mode in range(4):
        M, S = oracle.mttkrp(c, v, dims, A, mode)
        for r in range(world):
            got = out[r][0][mode]
            assert np.max(np.abs(got - M) / np.where(S > 0, S, 1)) <= 1e-12, (r, mode)


def test_partition_bounds():
    """blco_partition (host logic, no device): contiguous equal parts, inner
    bounds on multiples of 32, covering the store once."""
    import numpy as np

    from paper_2201_12523_gb300 import blco

    for nnz in (0, 1, 31, 32, 1000, 4099, 150_000_000):
        for parts in (1, 2, 3, 8, 152):
            b = blco.blco_partition(nnz, parts)
            assert b[0] == 0 and b[-1] == nnz and len(b) == parts + 1
            assert np.all(np.diff(b) >= 0)
            assert np.all(b[1:-1] % 32 == 0)
            if nnz >= 32 * parts * 4:
                sizes = np.diff(b)
                assert sizes.max() - sizes.min() <= 64
