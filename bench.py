"""All-mode sparse MTTKRP benchmark (one JSON line on rank 0).

Workload (default): the 3-mode skewed tensor 2^22 x 2^21 x 2^11 with 150M
distinct nonzeros, Zipf(1.2) indices with permuted labels, U(0,1) values,
rank 32, N(0,1) float32 factors -- synthetic, seeded, generated on the GPU.
A step is one all-mode MTTKRP (modes 0, 1, 2) over the BLCO store with
device-resident inputs; ``value`` is nonzeros processed per second per
all-mode step, summed over ranks. The store and factors (about 2.6 GB) are
larger than L2, so no flush is needed between steps.

Also reported: ``e2e`` (the same step through the C ABI with pinned host
factor matrices and host results, copies inside the timed region), the
bfloat16-factor variant, the roofline of the MTTKRP kernel (algorithmic bytes
per launch over its CUDA-event duration), the CPU baseline (the FP64 oracle
on a bounded sample), and SM clocks sampled during the timed region.

``--impl reference`` times the FP64 CPU oracle instead (rank 0 only).
Multi-GPU: independent replicas, one per rank (no collective on the data
path); the max time over ranks is used.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from paper_2201_12523_gb300 import synth  # noqa: E402

WORKLOADS = {s.name: s for s in synth.CONFIGS}
DEFAULT_WORKLOAD = "zipf1.2-3d-150M"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic of the MTTKRP kernel from an ncu capture (profiles/), valid only
# for the kernel source it was taken from (sha256 of csrc/mttkrp.cu).
TRAFFIC_RECORD = {"mttkrp_src_sha256": "90f9ba5c49e8fc275665fea7cdc21b875858ff1200bf1747bc38db028a0c50d3",
                  "bytes_per_launch": 4.493e9}  # mean of modes 0/1/2 at 150M nonzeros, R = 32, FP32


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=30)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="blco", choices=["blco", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-bf16", action="store_true")
    p.add_argument("--nnz", type=int, default=0, help="override the nonzero count (profiling captures only)")
    return p.parse_args(argv)


# ----------------------------------------------------------------- ranks
class Ranks:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if self.pg is None:
            return float(x)
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if self.pg is None:
            return float(x)
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()

    def rate(self, units: float, seconds: float) -> float:
        """Whole-job throughput: the units every rank processed over the
        slowest rank's time (each rank runs an independent replica)."""
        return self.sum(units) / self.max(seconds)


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def mttkrp_src_sha() -> str:
    """sha256 over the float32 MTTKRP kernel's sources (the kernel header and
    its translation unit), to tell whether a recorded ncu traffic figure
    still describes the kernel being timed."""
    h = hashlib.sha256()
    for name in ("mttkrp_kernels.cuh", "mttkrp_f32.cu"):
        with open(os.path.join(ROOT, "paper_2201_12523_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def algorithmic_bytes(spec, R: int, fbytes: int, mode: int, rows=None) -> int:
    """Compulsory bytes of one mode-n MTTKRP launch: the key/value stream
    (8 + 4 bytes per nonzero), every other factor matrix once, the output once.
    With `rows` (rows touched per mode) only the touched rows count: the
    stricter count."""
    rows = rows or spec.dims
    b = 12 * spec.nnz + 4 * rows[mode] * R
    for k, d in enumerate(rows):
        if k != mode:
            b += d * R * fbytes
    return b


def gen_inputs(spec, device):
    coords = synth.coordinates(spec, device=device)
    vals = synth.values(spec, device=device)
    A = synth.factors(spec, device=device)
    return coords, vals, A


# ----------------------------------------------------------------- CPU arms
def cpu_oracle_rate(spec, coords, vals, A, sample_nnz: int, repeats: int = 1):
    """The FP64 oracle, as it stands, on the first `sample_nnz` nonzeros of the
    workload (a random subset: the COO is in random order), all modes.
    Returns (nnz/s, seconds per step)."""
    import oracle

    oracle.build()
    c = coords[:sample_nnz].cpu().numpy().view(np.uint32)
    v = vals[:sample_nnz].cpu().numpy().astype(np.float64)
    Af = [a.cpu().numpy().astype(np.float64) for a in A]
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        for n in range(spec.order):
            oracle.mttkrp(c, v, spec.dims, Af, n)
        times.append(time.perf_counter() - t0)
    sec = statistics.median(times)
    return sample_nnz / sec, sec


def run_reference(args, ranks: Ranks):
    if ranks.rank != 0:
        return 0
    spec = WORKLOADS[args.workload]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    coords, vals, A = gen_inputs(spec, dev)
    sample = min(spec.nnz, 400_000)
    import oracle

    oracle.build()
    c = coords[:sample].cpu().numpy().astype(np.uint32)
    v = vals[:sample].cpu().numpy().astype(np.float64)
    Af = [a.cpu().numpy().astype(np.float64) for a in A]
    del coords, vals, A

    def step():
        for n in range(spec.order):
            oracle.mttkrp(c, v, spec.dims, Af, n)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    sec = (time.perf_counter() - t0) / max(args.steps, 1)
    value = sample / sec
    sample_desc = (f"first {sample} of the workload's {spec.nnz} nonzeros (random order), all "
                   f"{spec.order} modes per step, FP64, single thread")
    line = {"impl": "reference", "metric": "all-mode sparse MTTKRP throughput", "value": value,
            "unit": "nnz/s (all-mode)", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": spec.name, "rank": spec.rank},
            "cpu_baseline": {"value": value, "unit": "nnz/s (all-mode)", "cores": 1, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": "nnz/s (all-mode)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def time_steps(step, K: int, stream) -> float:
    """ms for K steps, CUDA events on the launching stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


CPU_SAMPLE_NNZ = 10_000_000  # oracle baseline sample: about 10 s of one core per all-mode pass
STREAMED = {"zipf1.2-5d-1B": 16 << 30}  # workloads run out of core: device budget in bytes
CP_MODEL = "cp-planted-3d-200M"


def host_link_gbs(dev, nbytes=2 << 30, reps=5) -> float:
    """Pinned host -> device copy bandwidth (GB/s), the out-of-memory bound."""
    src = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    dst.copy_(src, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        dst.copy_(src, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    gbs = nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
    del src, dst
    return gbs


def planted_store(blco, spec, coords, dev):
    """Store of the planted CP workload: values = the CP model of seeded U(0,1)
    factors at the coordinates (computed with the library's own forward kernel
    on a provisional store) plus N(0, 0.01) noise."""
    P = synth.factors(spec, device=dev, stream=5, dist="u01")
    tmp = blco.Tensor.build(coords, torch.zeros(coords.shape[0], device=dev), spec.dims)
    xhat = tmp.cp_fwd(P)
    perm = torch.from_numpy(tmp.perm()).to(dev)
    tmp.destroy()
    vals = torch.empty_like(xhat)
    vals[perm] = xhat
    vals += synth.noise(coords.shape[0], 0.01, spec.seed + 99, device=dev)
    del P, xhat, perm
    return vals


def run_blco(args, ranks: Ranks):
    from paper_2201_12523_gb300 import blco

    dev = torch.device("cuda", ranks.local)
    torch.cuda.set_device(dev)
    spec = WORKLOADS[args.workload]
    if args.nnz:
        spec = spec.scaled(args.nnz, spec.dims, name=f"{spec.name}@{args.nnz}")
    base_name = args.workload
    R = spec.rank
    t_gen = time.perf_counter()
    coords, vals, A = gen_inputs(spec, dev)
    if base_name == CP_MODEL:
        vals = planted_store(blco, spec, coords, dev)
        A = synth.factors(spec, device=dev, stream=1, dist="normal")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen
    torch.cuda.empty_cache()

    budget = STREAMED.get(base_name, 0)
    stream = torch.cuda.current_stream()
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    t = blco.Tensor.build(coords, vals, spec.dims, device_budget_bytes=budget, force_stream=bool(budget))
    eb1.record(stream)
    torch.cuda.synchronize()
    build_ms = eb0.elapsed_time(eb1)
    info = t.info()
    # rows each mode's nonzeros touch (for the stricter compulsory-bytes count)
    touched = [int(torch.unique(coords[:, n]).numel()) for n in range(spec.order)]
    # the same store with plain float32 run sums, for the bf16 comparison
    t_plain = None
    if not args.no_bf16 and not info["streamed"]:
        t_plain = blco.Tensor.build(coords, vals, spec.dims, plain_sums=True)
    coords_h = coords[: min(spec.nnz, CPU_SAMPLE_NNZ)].cpu()
    vals_h = vals[: min(spec.nnz, CPU_SAMPLE_NNZ)].cpu()
    del coords, vals
    torch.cuda.empty_cache()

    outs = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in spec.dims]

    if base_name == CP_MODEL:
        sv = t.values()
        grads = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in spec.dims]

        def make_step(factors, tt=None):
            tt = tt or t

            def step():
                # the sparse CP model at the nonzeros and the adjoint of a
                # least-squares loss for every factor (one kernel each)
                xhat = tt.cp_fwd(factors)
                g = xhat - sv
                for n in range(spec.order):
                    tt.cp_bwd(n, g, factors, out=grads[n])
            return step
        metric = "sparse CP forward + adjoint (all factors) throughput"
        kernel_kinds = ("mttkrp", "cp_fwd")
    else:
        def make_step(factors, tt=None):
            tt = tt or t

            def step():
                for n in range(spec.order):
                    tt.mttkrp(n, factors, out=outs[n])
            return step
        metric = "all-mode sparse MTTKRP throughput"
        kernel_kinds = ("mttkrp",)

    step32 = make_step(A)
    for _ in range(args.warmup):
        step32()
    torch.cuda.synchronize()

    sampler = ClockSampler(ranks.local)
    sampler.start()
    ranks.barrier()
    blco.blco_profile_enable(t.handle, True)
    ms = time_steps(step32, args.steps, stream)
    blco.blco_profile_enable(t.handle, False)
    prof = blco.blco_profile_read(t.handle)
    ranks.barrier()
    clocks = sampler.stop()
    ms_max = ranks.max(ms)
    ms_per_step = ms_max / args.steps
    value = ranks.rate(spec.nnz * args.steps, ms / 1e3)

    # roofline of the MTTKRP kernel: algorithmic bytes / mean launch duration
    peak, peak_src = hbm_peak()
    launches, kms = prof.get("mttkrp", (0, 0.0))
    zl, zms = prof.get("zero", (0, 0.0))
    fl, fms = prof.get("cp_fwd", (0, 0.0))
    sl, sms = prof.get("sum_copies", (0, 0.0))
    bytes_all = sum(algorithmic_bytes(spec, R, 4, n) for n in range(spec.order))
    per_launch_bytes = bytes_all / spec.order
    per_launch_ms = kms / max(launches, 1)
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9 if launches else None
    touched_bytes = sum(algorithmic_bytes(spec, R, 4, n, touched) for n in range(spec.order)) / spec.order
    traffic = None
    if TRAFFIC_RECORD["mttkrp_src_sha256"] == mttkrp_src_sha() and base_name == DEFAULT_WORKLOAD and not args.nnz:
        traffic = TRAFFIC_RECORD["bytes_per_launch"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel": f"k_mttkrp<float,{R},{spec.order - 1}>",
                "peak_source": peak_src + " (burst copy, MEASURED_PEAKS hbm_gbs)",
                "algorithmic_bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
                "touched_rows_per_mode": touched,
                "algorithmic_bytes_touched_rows": touched_bytes,
                "frac_touched_rows": (touched_bytes / (per_launch_ms / 1e3) / 1e9 / peak) if launches else None}
    if info["streamed"]:
        roofline["note"] = ("streamed store: kernel time measured on the queue streams; the step is bound by "
                            "the host link (see host_link)")

    extra = {}
    if info["streamed"]:
        link = host_link_gbs(dev)
        moved = 12 * spec.nnz * spec.order  # keys + values cross the link once per mode
        achieved_link = moved / (ms_per_step / 1e3) / 1e9
        ul, ums = prof.get("upload", (0, 0.0))
        extra["host_link"] = {"achieved": achieved_link, "peak": link, "unit": "GB/s",
                              "frac": achieved_link / link, "bytes_per_step": moved,
                              "upload_ms_per_step": ums / args.steps,
                              "upload_gbs_while_copying": moved * args.steps / (ums / 1e3) / 1e9 if ums else None,
                              "peak_source": "pinned cudaMemcpyAsync H2D, 2 GiB x 5, same run"}
        extra["store"] = "pinned host memory, %d queues x %d nonzeros, device budget %d GiB" % (
            info["n_queues"], info["queue_nnz"], budget >> 30)
    if base_name == CP_MODEL:
        extra["cp_fwd_ms_per_launch"] = fms / max(fl, 1)
        extra["adjoint_ms_per_launch"] = per_launch_ms
        Fals = synth.factors(spec, device=dev, stream=2, dist="u01")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, fits = blco.cp_als(t, Fals, iters=20)
        torch.cuda.synchronize()
        extra["cp_als"] = {"sweeps": 20, "s_per_sweep": (time.perf_counter() - t0) / 20,
                           "fit_first": fits[0], "fit_last": fits[-1],
                           "note": "MTTKRP in FP32, Gram Hadamard / Cholesky / fit in FP64 on the GPU"}
        del Fals

    # bfloat16 factors, same step
    if not args.no_bf16:
        A16 = [blco.convert(a, torch.bfloat16) for a in A]
        step16 = make_step(A16)
        for _ in range(args.warmup):
            step16()
        blco.blco_profile_enable(t.handle, True)
        ms16_local = time_steps(step16, args.steps, stream)
        ms16 = ranks.max(ms16_local)
        blco.blco_profile_enable(t.handle, False)
        p16 = blco.blco_profile_read(t.handle)
        l16, k16 = p16.get("mttkrp", (0, 0.0))
        b16 = sum(algorithmic_bytes(spec, R, 2, n) for n in range(spec.order)) / spec.order
        ach16 = b16 / (k16 / max(l16, 1) / 1e3) / 1e9 if l16 else None
        extra["bf16"] = {"value": ranks.rate(spec.nnz * args.steps, ms16_local / 1e3), "ms_per_step": ms16 / args.steps,
                         "speedup_vs_f32": ms_max / ms16, "roofline_frac": (ach16 / peak) if ach16 else None,
                         "run_sums": "Kahan-compensated",
                         "error_bound": 1e-2, "error_vs": "FP64 oracle on the unrounded float32 factors"}
        if t_plain is not None:
            stepp = make_step(A16, t_plain)
            for _ in range(args.warmup):
                stepp()
            msp_local = time_steps(stepp, args.steps, stream)
            msp = ranks.max(msp_local)
            extra["bf16_plain_sums"] = {"value": ranks.rate(spec.nnz * args.steps, msp_local / 1e3),
                                        "ms_per_step": msp / args.steps, "speedup_vs_f32": ms_max / msp,
                                        "run_sums": "plain float32 (build option plain_sums)"}
            t_plain.destroy()
        del A16

    # end to end through the C ABI with host buffers (MTTKRP workloads)
    e2e = None
    if not args.no_e2e and base_name != CP_MODEL:
        Ah = [a.cpu().pin_memory() for a in A]
        Oh = [torch.empty((d, R), dtype=torch.float32).pin_memory() for d in spec.dims]
        Ah_np = [a.numpy() for a in Ah]
        Oh_np = [o.numpy() for o in Oh]

        def step_e2e():
            blco.blco_mttkrp_all(t.handle, Ah_np, blco.BLCO_F32, R, Oh_np, stream)

        step_e2e()
        K2 = max(1, min(args.steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K2):
            step_e2e()
        torch.cuda.synchronize()
        sec_local = (time.perf_counter() - t0) / K2
        sec = ranks.max(sec_local)
        h2d = sum(d * R * 4 for d in spec.dims)
        d2h = h2d
        e2e = {"value": ranks.rate(spec.nnz, sec_local), "unit": "nnz/s (all-mode)", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": sec * 1e3, "steps": K2,
               "note": "blco_mttkrp_all with pinned host factors and host results; store built once"}

    cpu = None
    if not args.no_cpu and ranks.rank == 0:
        sample = min(spec.nnz, CPU_SAMPLE_NNZ)
        rate, sec = cpu_oracle_rate(spec, coords_h, vals_h, A, sample)
        cpu = {"value": rate, "unit": "nnz/s (all-mode)", "cores": 1, "kind": "oracle",
               "sample": f"first {sample} nonzeros of the workload (random order), all {spec.order} modes, "
                         f"FP64 C loops, one thread, {sec:.2f} s"}

    dists = sorted(set(spec.index_dist))
    line = {"metric": metric, "value": value, "unit": "nnz/s (all-mode)",
            "n_gpus": ranks.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": spec.name, "dims": list(spec.dims), "nnz": spec.nnz, "rank": R,
                       "factors": "float32 " + ("N(0,1)" if spec.factor_dist == "normal" or base_name == CP_MODEL
                                                 else "U(0,1)"),
                       "values": spec.value_dist if base_name != CP_MODEL else "planted rank-64 CP + N(0,0.01)",
                       "index_dist": ",".join(dists) + " (Zipf labels permuted)",
                       "parallelism": f"replicas x{ranks.world}",
                       "l2": "inputs larger than L2, no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches + zl + fl + sl),
            "build_ms": build_ms, "gen_s": gen_s,
            "construction": {"ms": build_ms, "nnz_per_s": spec.nnz / (build_ms / 1e3),
                             "all_mode_steps_to_amortize": build_ms / ms_per_step,
                             "note": "blco_build from device coordinates: linearize, radix sort, block, "
                                     "re-encode, hot-row histograms" + (", move to pinned host memory"
                                                                        if info["streamed"] else "")},
            "store": {"nblocks": info["nblocks"], "streamed": info["streamed"], "hot_rows": info["hot_rows"],
                      "device_bytes": info["device_bytes"]}}
    line.update(extra)
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
    t.destroy()
    return 0


def main(argv=None):
    args = parse_args(argv)
    ranks = Ranks()
    try:
        if args.impl == "reference":
            return run_reference(args, ranks)
        return run_blco(args, ranks)
    finally:
        ranks.close()


if __name__ == "__main__":
    sys.exit(main())
