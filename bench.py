"""All-mode sparse MTTKRP benchmark (one JSON line on rank 0).

Headline workload (the largest in-memory configuration, the one the metric's
"BF16 vs FP32 at stated error" is quoted on): the 4-mode skewed tensor
2^20 x 2^18 x 2^16 x 2^8 with 500M distinct nonzeros, Zipf(1.1) indices with
permuted labels, lognormal(0,1) values, rank 32, N(0,1) float32 factors --
synthetic, seeded, generated on the GPU. A step is one all-mode MTTKRP
(modes 0..3) over the BLCO store with device-resident inputs; ``value`` is
nonzeros processed per second per all-mode step, summed over ranks. The
store and factors (about 6 GB) are larger than L2, so no flush is needed
between steps.

Also reported on the headline workload: ``e2e`` (the same step through the C
ABI with pinned host factor matrices and host results, copies inside the
timed region), the bfloat16-factor step with its speedup and its measured
error per mode against the FP64 oracle (sampled heavy and random output
rows; against the unrounded and the bf16-rounded factors; the float32 errors
beside them), the roofline of the MTTKRP kernel (algorithmic bytes per launch
over its CUDA-event duration), the CPU baseline (the FP64 oracle on a
bounded sample, on all host cores and on one), and SM clocks sampled during
the timed region. ``workloads`` carries the other three large workloads,
measured in the same run: the 3-mode 150M tensor, the 5-mode 1B tensor
streamed from pinned host memory under a 16 GiB device budget (host-link
fraction), and the planted-CP 200M tensor (forward + adjoint, 20 CP-ALS
sweeps).

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
DEFAULT_WORKLOAD = "zipf1.1-4d-500M"
EXTRA_WORKLOADS = ("zipf1.2-3d-150M", "zipf1.2-5d-1B", "cp-planted-3d-200M")
STREAMED = {"zipf1.2-5d-1B": 16 << 30}  # workloads run out of core: device budget in bytes
CP_MODEL = "cp-planted-3d-200M"
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FP32_TOL, BF16_TOL = 1e-5, 1e-2

# DRAM traffic of the MTTKRP kernel per launch from one ncu capture
# (profiles/), valid only for the kernel source it was taken from (sha256 of
# the kernel header and its float32 translation unit): workload -> record.
TRAFFIC_RECORDS = {
    "zipf1.1-4d-500M": {"src_sha256": "e6765c8922a7d71eafc404c1d1ce06398280425ae954f857e53e8aeec58b933b",
                        "bytes_per_launch": 7.223e9},  # mean of modes 0-3, R = 32, float32 factors
    "zipf1.2-5d-1B": {"src_sha256": "c16df474c0ced002e24fc1c056d4e7cee614803c50b329a74341cd539b008162",
                      "bytes_per_launch": 28.785e9},  # one-pass all-mode launch, resident store, R = 16
}


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="blco", choices=["blco", "reference"])
    p.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                   help="measure this workload alone (default: the headline workload plus the other three)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-bf16", action="store_true")
    p.add_argument("--no-errors", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--f64", action="store_true",
                   help="with --workload: also time the float64 path (values, factors, accumulation)")
    p.add_argument("--nnz", type=int, default=0, help="override the nonzero count (profiling captures only)")
    p.add_argument("--resident", action="store_true",
                   help="keep the store on the device for a workload that streams (profiling captures only)")
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

    def _reduce(self, x: float, op) -> float:
        if self.pg is None:
            return float(x)
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, self.pg.ReduceOp.MAX if self.pg else None)

    def sum(self, x: float) -> float:
        return self._reduce(x, self.pg.ReduceOp.SUM if self.pg else None)

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


def mttkrp_src_sha(onepass: bool = False) -> str:
    """sha256 over the MTTKRP kernel's sources (the kernel header and the
    float32 translation unit, or the one-pass kernel's unit), to tell whether
    a recorded ncu traffic figure still describes the kernel being timed."""
    h = hashlib.sha256()
    for name in ("mttkrp_kernels.cuh", "mttkrp_fused.cu" if onepass else "mttkrp_f32.cu"):
        with open(os.path.join(ROOT, "paper_2201_12523_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def algorithmic_bytes(spec, R: int, fbytes: int, mode: int, rows=None) -> int:
    """Compulsory bytes of one mode-n MTTKRP launch: the key/value stream
    (8 + 4 bytes per nonzero), every other factor matrix once (fbytes per
    entry), the float32 output once. With `rows` (rows touched per mode) only
    the touched rows count: the stricter count."""
    rows = rows or spec.dims
    b = 12 * spec.nnz + 4 * rows[mode] * R
    for k, d in enumerate(rows):
        if k != mode:
            b += d * R * fbytes
    return b


def onepass_bytes(spec, R: int, fbytes: int, rows=None) -> int:
    """Compulsory bytes of one all-mode launch of the one-pass kernel (5-mode
    stores): the key/value stream once, every factor matrix once, every
    float32 output once."""
    rows = rows or spec.dims
    return 12 * spec.nnz + sum(d * R * (fbytes + 4) for d in rows)


def mttkrp_kind(prof) -> str:
    """Profile kind of the MTTKRP kernel an all-mode step ran: the one-pass
    kernel (5-mode stores) or the per-mode kernel."""
    return "mttkrp_all_fused" if prof.get("mttkrp_all_fused", (0, 0.0))[0] else "mttkrp"


def gen_inputs(spec, device):
    coords = synth.coordinates(spec, device=device)
    vals = synth.values(spec, device=device)
    A = synth.factors(spec, device=device)
    return coords, vals, A


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
    """Values of the planted CP workload: the CP model of seeded U(0,1)
    factors at the coordinates (the library's own forward kernel on a
    provisional store) plus N(0, 0.01) noise."""
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


def kernel_roofline(prof, kind, bytes_per_launch, peak):
    launches, kms = prof.get(kind, (0, 0.0))
    if not launches:
        return None, None, 0
    ms = kms / launches
    ach = bytes_per_launch / (ms / 1e3) / 1e9
    return ach, ms, launches


# ----------------------------------------------------------------- oracle legs (CPU)
def cpu_baseline_leg(spec, c_h, v_h, A):
    """The FP64 oracle, as it stands, timed on this host's cores over a
    bounded sample of the workload (the first nonzeros of the COO, which is
    in random order): all cores with the row-parallel mttkrp_rows over every
    output row, and one core with the plain loop of mttkrp. Returns
    (all-core line, one-core line)."""
    import oracle

    oracle.build()
    Af = [a.cpu().numpy().astype(np.float64) for a in A]
    cores = os.cpu_count() or 1
    lines = []
    for label, sample, fn in (("all cores", 50_000_000, "rows"), ("one core", 5_000_000, "plain")):
        n = min(spec.nnz, sample, c_h.shape[0])
        c = c_h[:n]
        v = v_h[:n].astype(np.float64)
        t0 = time.perf_counter()
        for m in range(spec.order):
            if fn == "rows":
                oracle.mttkrp_rows(c, v, spec.dims, Af, m, np.arange(spec.dims[m]))
            else:
                oracle.mttkrp(c, v, spec.dims, Af, m)
        sec = time.perf_counter() - t0
        lines.append({"value": n / sec, "unit": "nnz/s (all-mode)", "cores": cores if fn == "rows" else 1,
                      "kind": "oracle",
                      "sample": f"first {n} of the workload's {spec.nnz} nonzeros (random order), all "
                                f"{spec.order} modes, FP64 C loops ({'OpenMP over output rows, ' + str(cores) + ' threads' if fn == 'rows' else 'one thread'}), {sec:.2f} s"})
    return lines[0], lines[1]


def rows_to_check(c_h, dims, seed, n_top=8, n_rand=24):
    rng = np.random.default_rng(seed)
    out = []
    for n, I in enumerate(dims):
        counts = np.bincount(np.ascontiguousarray(c_h[:, n]), minlength=I)
        top = np.argsort(counts)[::-1][:n_top]
        rand = rng.choice(I, size=min(n_rand, I), replace=False)
        out.append(np.unique(np.concatenate([top, rand])))
    return out


def error_leg(spec, c_h, v_h, A, results):
    """Measured max relative error per mode (max |M - M_ref| / sum |terms|)
    of the GPU results against the FP64 oracle, on the heaviest and random
    output rows of every mode. `results` maps a label to (per-mode outputs
    restricted to those rows, reference kind: 'f32' = the float32 factors,
    'bf16' = the same factors rounded to bfloat16)."""
    import oracle

    oracle.build()
    rows = rows_to_check(c_h, spec.dims, 5)
    v64 = v_h.astype(np.float64)
    refs = {}
    Af = [a.cpu().numpy().astype(np.float64) for a in A]
    refs["f32"] = Af
    if any(kind == "bf16" for _, kind in results.values()):
        refs["bf16"] = [oracle.bf16_round(a.cpu().numpy()).astype(np.float64) for a in A]
    cache = {}
    out = {}
    for label, (outs, kind) in results.items():
        errs = []
        for n in range(spec.order):
            if (kind, n) not in cache:
                cache[(kind, n)] = oracle.mttkrp_rows(c_h, v64, spec.dims, refs[kind], n, rows[n])
            M, S = cache[(kind, n)]
            errs.append(oracle.max_rel_err(outs[n](rows[n]), M, S))
        out[label] = errs
    return out, [int(len(r)) for r in rows]


# ----------------------------------------------------------------- reference arm
def run_reference(args, ranks: Ranks):
    if ranks.rank != 0:
        return 0
    spec = WORKLOADS[args.workload or DEFAULT_WORKLOAD]
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    coords, vals, A = gen_inputs(spec, dev)
    # a bounded sample per step, the oracle's row-parallel form on all cores
    # (as the main line's cpu_baseline): one to two seconds per step on 16 cores
    sample = min(spec.nnz, 8_000_000)
    import oracle

    oracle.build()
    c = coords[:sample].cpu().numpy().astype(np.uint32)
    v = vals[:sample].cpu().numpy().astype(np.float64)
    Af = [a.cpu().numpy().astype(np.float64) for a in A]
    del coords, vals, A

    all_rows = [np.arange(d) for d in spec.dims]
    cores = os.cpu_count() or 1

    def step():
        for n in range(spec.order):
            oracle.mttkrp_rows(c, v, spec.dims, Af, n, all_rows[n])

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    sec = (time.perf_counter() - t0) / max(args.steps, 1)
    value = sample / sec
    sample_desc = (f"first {sample} of the workload's {spec.nnz} nonzeros (random order), all "
                   f"{spec.order} modes per step, FP64 C loops (OpenMP over output rows, {cores} threads)")
    line = {"impl": "reference", "metric": "all-mode sparse MTTKRP throughput", "value": value,
            "unit": "nnz/s (all-mode)", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "config": {"workload": spec.name, "rank": spec.rank},
            "cpu_baseline": {"value": value, "unit": "nnz/s (all-mode)", "cores": cores, "kind": "oracle",
                             "sample": sample_desc},
            "e2e": {"value": value, "unit": "nnz/s (all-mode)", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm
def measure_mttkrp(blco, spec, args, ranks, dev, steps, warmup, *, headline, sampler=None, with_f64=False):
    """All-mode MTTKRP of an in-memory or streamed workload. Returns a dict
    (and the headline keys when `headline`)."""
    R = spec.rank
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    coords, vals, A = gen_inputs(spec, dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen
    torch.cuda.empty_cache()
    budget = 0 if args.resident else STREAMED.get(spec.name.split("@")[0], 0)
    eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eb0.record(stream)
    t = blco.Tensor.build(coords, vals, spec.dims, device_budget_bytes=budget, force_stream=bool(budget))
    eb1.record(stream)
    torch.cuda.synchronize()
    build_ms = eb0.elapsed_time(eb1)
    info = t.info()
    touched = [int(torch.unique(coords[:, n]).numel()) for n in range(spec.order)]
    want_bf16 = not args.no_bf16 and not info["streamed"]
    t_comp = blco.Tensor.build(coords, vals, spec.dims, compensated_sums=True) if (want_bf16 and headline) else None
    t64 = blco.Tensor.build(coords, vals.double(), spec.dims) if with_f64 else None
    # a streamed workload is also timed on a store resident on the device: the
    # same all-mode MTTKRP without the host link
    t_res = blco.Tensor.build(coords, vals, spec.dims) if info["streamed"] else None
    # ... and on a streamed store whose kernels read it in pinned host memory
    # (build option host_reads: no device queues or batch copies)
    t_hr = (blco.Tensor.build(coords, vals, spec.dims, device_budget_bytes=budget, force_stream=True, host_reads=True)
            if info["streamed"] else None)
    need_host = headline and (not args.no_errors or not args.no_cpu) and ranks.rank == 0
    c_h = coords.cpu().numpy().view(np.uint32) if need_host else None
    v_h = vals.cpu().numpy() if need_host else None
    del coords, vals
    torch.cuda.empty_cache()

    outs = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in spec.dims]

    def make_step(factors, tt, o):
        def step():
            tt.mttkrp_all(factors, outs=o)  # one C-ABI call: every mode's MTTKRP
        return step

    step32 = make_step(A, t, outs)
    for _ in range(warmup):
        step32()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ranks.barrier()
    blco.blco_profile_enable(t.handle, True)
    ms = time_steps(step32, steps, stream)
    blco.blco_profile_enable(t.handle, False)
    prof = blco.blco_profile_read(t.handle)
    ranks.barrier()
    clocks = sampler.stop() if sampler else None
    ms_max = ranks.max(ms)
    res = {"workload": spec.name, "nnz": spec.nnz, "rank": R, "steps": steps, "warmup": warmup,
           "ms_per_step": ms_max / steps, "value": ranks.rate(spec.nnz * steps, ms / 1e3),
           "unit": "nnz/s (all-mode)", "gen_s": gen_s}
    peak, peak_src = hbm_peak()
    kind = mttkrp_kind(prof)
    onepass = kind == "mttkrp_all_fused"
    if onepass:
        b32 = onepass_bytes(spec, R, 4)
        touched_bytes = onepass_bytes(spec, R, 4, touched)
        kname = f"k_mttkrp_fused<float,{R},{spec.order}>"
    else:
        b32 = sum(algorithmic_bytes(spec, R, 4, n) for n in range(spec.order)) / spec.order
        touched_bytes = sum(algorithmic_bytes(spec, R, 4, n, touched) for n in range(spec.order)) / spec.order
        kname = f"k_mttkrp<float,{R},{spec.order - 1}>"
    ach, kms, kl = kernel_roofline(prof, kind, b32, peak)
    rec = TRAFFIC_RECORDS.get(spec.name)
    traffic = rec["bytes_per_launch"] if rec and rec["src_sha256"] == mttkrp_src_sha(onepass) else None
    res["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                       "frac": (ach / peak) if ach else None, "traffic": traffic,
                       "kernel": kname,
                       "launch": "one launch per all-mode step (every mode in one pass)" if onepass
                       else "one launch per mode",
                       "peak_source": peak_src + " (burst copy, MEASURED_PEAKS hbm_gbs)",
                       "algorithmic_bytes_per_launch": b32, "ms_per_launch": kms,
                       "touched_rows_per_mode": touched, "algorithmic_bytes_touched_rows": touched_bytes,
                       "frac_touched_rows": (touched_bytes / (kms / 1e3) / 1e9 / peak) if kms else None}
    zl = prof.get("zero", (0, 0.0))[0]
    sl = prof.get("sum_copies", (0, 0.0))[0]
    res["gpu_launches"] = int(kl + zl + sl)
    res["clocks"] = clocks
    res["construction"] = {"ms": build_ms, "nnz_per_s": spec.nnz / (build_ms / 1e3),
                           "all_mode_steps_to_amortize": build_ms / res["ms_per_step"],
                           "note": "blco_build from device coordinates: linearize, radix sort, block, re-encode, "
                                   "hot-row histograms" + (", move to pinned host memory" if info["streamed"] else "")}
    res["store"] = {"nblocks": info["nblocks"], "streamed": info["streamed"], "hot_rows": info["hot_rows"],
                    "device_bytes": info["device_bytes"], "host_bytes": info["host_bytes"]}
    if info["streamed"]:
        res["roofline"]["note"] = "streamed store: see host_link; the kernel roofline is taken on a resident copy"
        link = host_link_gbs(dev)
        ul, ums = prof.get("upload", (0, 0.0))
        moved = 12 * spec.nnz  # keys + values cross the link once per all-mode step
        achieved_link = moved / (res["ms_per_step"] / 1e3) / 1e9
        res["host_link"] = {"achieved": achieved_link, "peak": link, "unit": "GB/s", "frac": achieved_link / link,
                            "bytes_per_step": moved, "upload_ms_per_step": ums / steps,
                            "upload_gbs_while_copying": moved * steps / (ums / 1e3) / 1e9 if ums else None,
                            "peak_source": "pinned cudaMemcpyAsync H2D, 2 GiB x 5, same run"}
        res["store"]["queues"] = f"{info['n_queues']} queues x {info['queue_nnz']} nonzeros, device budget " \
                                 f"{budget >> 30} GiB"
        outs_r = [torch.empty_like(o) for o in outs]
        step_r = make_step(A, t_res, outs_r)
        for _ in range(warmup):
            step_r()
        blco.blco_profile_enable(t_res.handle, True)
        ms_r = ranks.max(time_steps(step_r, steps, stream)) / steps
        blco.blco_profile_enable(t_res.handle, False)
        ach_r, kms_r, _ = kernel_roofline(blco.blco_profile_read(t_res.handle), kind, b32, peak)
        if ach_r:
            # batches of the streamed store overlap on the queue streams, so their
            # launch durations say little; a resident launch covers the whole store
            res["roofline"].update({"achieved": ach_r, "frac": ach_r / peak, "ms_per_launch": kms_r,
                                    "frac_touched_rows": touched_bytes / (kms_r / 1e3) / 1e9 / peak,
                                    "streamed_batch_ms_per_launch": kms})
        t_res.destroy()
        t_res = None
        del outs_r
        link_ms = moved / (link * 1e9) * 1e3
        res["host_link"]["resident_ms_per_step"] = ms_r
        res["host_link"]["link_ms_per_step_at_peak"] = link_ms
        res["host_link"]["bound"] = ("kernels: the all-mode MTTKRP of a resident store takes %.0f ms, longer than "
                                     "the %.0f ms the host link needs for the store at its measured peak" % (ms_r, link_ms)
                                     if ms_r > link_ms else "host link")
        # the same step with the kernel reading the store in host memory
        outs_h = [torch.empty_like(o) for o in outs]
        step_h = make_step(A, t_hr, outs_h)
        for _ in range(warmup):
            step_h()
        ms_h = ranks.max(time_steps(step_h, steps, stream)) / steps
        ih = t_hr.info()
        ach_h = moved / (ms_h / 1e3) / 1e9
        res["host_reads"] = {"ms_per_step": ms_h, "value": ranks.rate(spec.nnz, ms_h / 1e3),
                             "unit": "nnz/s (all-mode)", "host_link_achieved": ach_h, "host_link_frac": ach_h / link,
                             "device_bytes": ih["device_bytes"], "host_bytes": ih["host_bytes"],
                             "note": "build option host_reads: one all-mode launch loads the store's keys and values "
                                     "from pinned host memory over the host link; no device queues or batch copies"}
        t_hr.destroy()
        t_hr = None
        del outs_h

    # bfloat16 factors, same step; Kahan-compensated run sums on the second store
    err_results = {}
    if want_bf16:
        A16 = [blco.convert(a, torch.bfloat16) for a in A]
        outs16 = [torch.empty_like(o) for o in outs]
        step16 = make_step(A16, t, outs16)
        for _ in range(warmup):
            step16()
        blco.blco_profile_enable(t.handle, True)
        ms16 = ranks.max(time_steps(step16, steps, stream))
        blco.blco_profile_enable(t.handle, False)
        p16 = blco.blco_profile_read(t.handle)
        b16 = onepass_bytes(spec, R, 2) if onepass else \
            sum(algorithmic_bytes(spec, R, 2, n) for n in range(spec.order)) / spec.order
        ach16, kms16, _ = kernel_roofline(p16, kind, b16, peak)
        res["bf16"] = {"value": ranks.rate(spec.nnz * steps, ms16 / 1e3), "ms_per_step": ms16 / steps,
                       "speedup_vs_f32": ms_max / ms16, "ms_per_launch": kms16,
                       "roofline_frac": (ach16 / peak) if ach16 else None,
                       "run_sums": "plain float32 (the default)",
                       "error_bound": {"vs_unrounded_f32_factors": BF16_TOL, "vs_bf16_rounded_factors": FP32_TOL}}
        err_results["bf16"] = (outs16, "bf16")
        if t_comp is not None:
            outsc = [torch.empty_like(o) for o in outs]
            stepc = make_step(A16, t_comp, outsc)
            for _ in range(warmup):
                stepc()
            msc = ranks.max(time_steps(stepc, steps, stream))
            res["bf16_compensated_sums"] = {"value": ranks.rate(spec.nnz * steps, msc / 1e3),
                                            "ms_per_step": msc / steps, "speedup_vs_f32": ms_max / msc,
                                            "run_sums": "Kahan-compensated (build option compensated_sums)"}
            err_results["bf16_compensated_sums"] = (outsc, "bf16")
            t_comp.destroy()
            t_comp = None
        del A16
    err_results["f32"] = (outs, "f32")

    # float64 values, factors and accumulation (the paper's precision), same step
    if t64 is not None:
        A64 = [a.double() for a in A]
        outs64 = [torch.empty((d, R), dtype=torch.float64, device=dev) for d in spec.dims]

        def step64():
            for n in range(spec.order):
                t64.mttkrp_f64(n, A64, out=outs64[n])
        for _ in range(warmup):
            step64()
        blco.blco_profile_enable(t64.handle, True)
        ms64 = ranks.max(time_steps(step64, steps, stream))
        blco.blco_profile_enable(t64.handle, False)
        p64 = blco.blco_profile_read(t64.handle)
        b64 = sum(16 * spec.nnz + 8 * R * sum(spec.dims) for _ in range(spec.order)) / spec.order
        ach64, kms64, _ = kernel_roofline(p64, "mttkrp_f64", b64, peak)
        res["f64"] = {"value": ranks.rate(spec.nnz * steps, ms64 / 1e3), "ms_per_step": ms64 / steps,
                      "ms_per_launch": kms64, "roofline_frac": (ach64 / peak) if ach64 else None,
                      "algorithmic_bytes_per_launch": b64, "speedup_vs_f32": ms_max / ms64,
                      "note": "float64 values, factors, accumulation and output (blco_mttkrp_f64)"}
        t64.destroy()
        del A64, outs64

    # end to end through the C ABI with host buffers
    if headline and not args.no_e2e:
        Ah = [a.cpu().pin_memory() for a in A]
        Oh = [torch.empty((d, R), dtype=torch.float32).pin_memory() for d in spec.dims]
        Ah_np = [a.numpy() for a in Ah]
        Oh_np = [o.numpy() for o in Oh]

        def step_e2e():
            blco.blco_mttkrp_all(t.handle, Ah_np, blco.BLCO_F32, R, Oh_np, stream)

        step_e2e()
        K2 = max(1, min(steps, 10))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K2):
            step_e2e()
        torch.cuda.synchronize()
        sec_local = (time.perf_counter() - t0) / K2
        sec = ranks.max(sec_local)
        h2d = sum(d * R * 4 for d in spec.dims)
        res["e2e"] = {"value": ranks.rate(spec.nnz, sec_local), "unit": "nnz/s (all-mode)",
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d, "ms_per_step": sec * 1e3, "steps": K2,
                      "note": "blco_mttkrp_all with pinned host factors and host results; store built once"}
        del Ah, Oh

    if need_host and not args.no_errors:
        t0 = time.perf_counter()
        sel = {}
        for label, (o, kind) in err_results.items():
            sel[label] = ([(lambda rows, x=x: x[torch.from_numpy(rows).to(dev)].cpu().numpy()) for x in o], kind)
        if "bf16" in sel:  # the bf16 outputs also against the oracle on the unrounded float32 factors
            sel["bf16_unrounded"] = (sel["bf16"][0], "f32")
        errs, nrows = error_leg(spec, c_h, v_h, A, sel)
        res["errors"] = {"metric": "max_{i,r} |M - M_ref| / sum |x prod a| per mode, FP64 oracle",
                         "rows_per_mode": nrows, "rows": "8 heaviest + 24 random output rows per mode",
                         "f32_vs_f32_factors": errs.get("f32")}
        if "bf16" in errs:
            res["errors"]["bf16_vs_unrounded_f32_factors"] = errs["bf16_unrounded"]
            res["errors"]["bf16_vs_bf16_rounded_factors"] = errs["bf16"]
            if "bf16_compensated_sums" in errs:
                res["errors"]["bf16_compensated_sums_vs_bf16_rounded_factors"] = errs["bf16_compensated_sums"]
        res["errors"]["oracle_s"] = time.perf_counter() - t0
        if "bf16" in res:
            res["bf16"]["error_per_mode"] = {
                "vs_unrounded_f32_factors": res["errors"].get("bf16_vs_unrounded_f32_factors"),
                "vs_bf16_rounded_factors": res["errors"].get("bf16_vs_bf16_rounded_factors"),
                "f32_factors_vs_f32": res["errors"]["f32_vs_f32_factors"]}
    if need_host and not args.no_cpu:
        res["cpu_baseline"], res["cpu_baseline_one_core"] = cpu_baseline_leg(spec, c_h, v_h, A)
    t.destroy()
    del outs, A
    torch.cuda.empty_cache()
    return res


def measure_cp(blco, spec, args, ranks, dev, steps, warmup):
    """Sparse CP forward + adjoint of every factor (float32 and bfloat16
    factors) and 20 CP-ALS sweeps on the planted workload."""
    R = spec.rank
    stream = torch.cuda.current_stream()
    t_gen = time.perf_counter()
    coords = synth.coordinates(spec, device=dev)
    vals = planted_store(blco, spec, coords, dev)
    A = synth.factors(spec, device=dev, stream=1, dist="normal")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen
    t = blco.Tensor.build(coords, vals, spec.dims)
    del coords, vals
    torch.cuda.empty_cache()
    sv = t.values()
    grads = [torch.empty((d, R), dtype=torch.float32, device=dev) for d in spec.dims]

    def make_step(factors):
        def step():
            xhat = t.cp_fwd(factors)
            g = xhat - sv
            for n in range(spec.order):
                t.cp_bwd(n, g, factors, out=grads[n])
        return step

    res = {"workload": spec.name, "nnz": spec.nnz, "rank": R, "steps": steps, "gen_s": gen_s,
           "metric": "sparse CP forward + adjoint (all factors) throughput", "unit": "nnz/s"}
    peak, _ = hbm_peak()
    for label, factors, fb in (("f32", A, 4), ("bf16", [blco.convert(a, torch.bfloat16) for a in A], 2)):
        step = make_step(factors)
        for _ in range(warmup):
            step()
        blco.blco_profile_enable(t.handle, True)
        ms = ranks.max(time_steps(step, steps, stream))
        blco.blco_profile_enable(t.handle, False)
        prof = blco.blco_profile_read(t.handle)
        badj = sum(algorithmic_bytes(spec, R, fb, n) for n in range(spec.order)) / spec.order
        bfwd = 16 * spec.nnz + sum(d * R * fb for d in spec.dims)
        ach_a, ms_a, _ = kernel_roofline(prof, "mttkrp", badj, peak)
        ach_f, ms_f, _ = kernel_roofline(prof, "cp_fwd", bfwd, peak)
        res[label] = {"ms_per_step": ms / steps, "value": ranks.rate(spec.nnz * steps, ms / 1e3),
                      "adjoint_ms_per_launch": ms_a, "adjoint_roofline_frac": ach_a / peak if ach_a else None,
                      "cp_fwd_ms_per_launch": ms_f, "cp_fwd_roofline_frac": ach_f / peak if ach_f else None}
    res["bf16"]["speedup_vs_f32"] = res["f32"]["ms_per_step"] / res["bf16"]["ms_per_step"]
    Fals = synth.factors(spec, device=dev, stream=2, dist="u01")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, fits = blco.cp_als(t, Fals, iters=20)
    torch.cuda.synchronize()
    res["cp_als"] = {"sweeps": 20, "s_per_sweep": (time.perf_counter() - t0) / 20, "fit_first": fits[0],
                     "fit_last": fits[-1],
                     "note": "MTTKRP in FP32, Gram Hadamard / Cholesky / fit in FP64 on the GPU"}
    t.destroy()
    del A, Fals, grads, sv
    torch.cuda.empty_cache()
    return res


def run_blco(args, ranks: Ranks):
    from paper_2201_12523_gb300 import blco

    dev = torch.device("cuda", ranks.local)
    torch.cuda.set_device(dev)
    name = args.workload or DEFAULT_WORKLOAD
    spec = WORKLOADS[name]
    if args.nnz:
        spec = spec.scaled(args.nnz, spec.dims, name=f"{spec.name}@{args.nnz}")
    sampler = ClockSampler(ranks.local)
    if name == CP_MODEL:
        head = measure_cp(blco, spec, args, ranks, dev, args.steps, args.warmup)
        head["clocks"] = None
        head["value"] = head["f32"]["value"]
        head["ms_per_step"] = head["f32"]["ms_per_step"]
        metric = head.pop("metric")
        roof = None
    else:
        head = measure_mttkrp(blco, spec, args, ranks, dev, args.steps, args.warmup, headline=True,
                              sampler=sampler, with_f64=args.f64 and spec.name.split("@")[0] not in STREAMED)
        metric = "all-mode sparse MTTKRP throughput"
        roof = head.pop("roofline")
    line = {"metric": metric, "value": head.pop("value"), "unit": head.pop("unit", "nnz/s (all-mode)"),
            "n_gpus": ranks.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head.pop("ms_per_step", None), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": spec.name, "dims": list(spec.dims), "nnz": spec.nnz, "rank": spec.rank,
                       "factors": "float32 " + ("N(0,1)" if spec.factor_dist == "normal" or name == CP_MODEL
                                                 else "U(0,1)"),
                       "values": spec.value_dist if name != CP_MODEL else "planted rank-64 CP + N(0,0.01)",
                       "index_dist": ",".join(sorted(set(spec.index_dist))) + " (Zipf labels permuted)",
                       "parallelism": f"replicas x{ranks.world}", "l2": "inputs larger than L2, no flush"},
            "roofline": roof, "cpu_baseline": head.pop("cpu_baseline", None), "e2e": head.pop("e2e", None),
            "clocks": head.pop("clocks", None), "gpu_launches": head.pop("gpu_launches", None)}
    line.update(head)
    if args.workload is None and not args.no_extras and ranks.world == 1 and not args.nnz:
        line["workloads"] = {}
        for extra in EXTRA_WORKLOADS:
            es = WORKLOADS[extra]
            t0 = time.perf_counter()
            if extra == CP_MODEL:
                r = measure_cp(blco, es, args, ranks, dev, 5, 3)
            else:
                streamed = extra in STREAMED
                r = measure_mttkrp(blco, es, args, ranks, dev, 3 if streamed else 10, 2 if streamed else 3,
                                   headline=False, with_f64=not streamed)
            r["wall_s"] = time.perf_counter() - t0
            line["workloads"][extra] = r
    if ranks.rank == 0:
        print(json.dumps(line), flush=True)
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
