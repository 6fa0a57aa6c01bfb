"""Benchmark of the GB300 PIR first-dimension scan.

One step = one pir_answer of one batch of B query ciphertext sets against a
resident NTT-form database: forward NTT of the queries, the per-slot modular
GEMM with its reduction, and the inverse NTT of the responses.  The metric is
DB-scan throughput in raw DB bytes x queries / s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--batch B]
                  [--layout plain|limb|tensor] [--impl ours|reference] [--noalloc]
  python bench.py --serving | --ntt-sweep | --lwe       (the other measurements)

With no flags the line is the 16 GiB database (n = 4096, 4096 x 512) at batch 32 on
the exact integer plain path, plus blocks at batches 1, 8 and 128 (`per_batch`), the
tensor layout at batch 32 (`tensor_layout`), and the 32 GiB database at batch 64 on
the plain and limb layouts (`largest_config`), each timed for at least a second.

Prints one JSON line (rank 0).  Under torchrun (N > 1) every rank holds its own
replica of the database and answers its own batches (independent problems, no
data-path collective); the value is the queries of all ranks over the slowest
rank's time.  ``--impl reference`` times the CPU oracle instead (the only other
place this file runs it, besides the cpu_baseline leg).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DB-scan GB/s (raw DB bytes×queries/s) at batch 1..128; serving p50/p99 ms"

# name -> (n, log2p, D1, D2, default batch, description)
WORKLOADS = {
    "tiny_n2048": (2048, 12, 16, 16, 1, "768 KiB raw DB, n=2048, p=2^12, 16x16 polys"),
    "db1g_n4096": (4096, 16, 512, 256, 1, "1 GiB raw DB (4 GiB NTT-form), n=4096, p=2^16, D1=512, D2=256"),
    "db256m_n4096": (4096, 16, 128, 256, 1, "256 MiB raw DB (1 GiB NTT-form), n=4096, p=2^16, D1=128, D2=256"),
    "db512m_n2048": (2048, 16, 512, 256, 1, "512 MiB raw DB (2 GiB NTT-form), n=2048, p=2^16, D1=512, D2=256"),
    "db1g_n2048": (2048, 16, 512, 512, 1, "1 GiB raw DB (4 GiB NTT-form), n=2048, p=2^16, D1=512, D2=512"),
    "db8g_n4096": (4096, 16, 2048, 512, 1, "8 GiB raw DB (32 GiB NTT-form), n=4096, p=2^16, D1=2048, D2=512"),
    "db16g_n4096": (4096, 16, 4096, 512, 32, "16 GiB raw DB (64 GiB NTT-form), n=4096, p=2^16, D1=4096, D2=512"),
    "db32g_n8192": (8192, 16, 8192, 256, 64, "32 GiB raw DB (128 GiB NTT-form), n=8192, p=2^16, D1=8192, D2=256"),
}
DEFAULT_WORKLOAD = "db16g_n4096"
PER_BATCH = (1, 8, 32, 128)  # the metric's batch range
MIN_TIMED_S = 1.0  # each extra block times at least this long
L_PRIMES = 2
FALLBACK_HBM_GBS = 6800.0


def sha256_of(path: str) -> str:
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def profile_traffic(kernel_tag: str, workload: str, batch: int, source: str, launches_per_step: float = None):
    """Per-launch DRAM bytes of a kernel from a committed ncu summary, or None when
    there is none for this workload, the kernel source changed since, or the summary
    names a number of launches per step (K-chunks) other than the timed one's."""
    path = os.path.join(ROOT, "profiles", "%s_%s_b%d.txt" % (kernel_tag, workload, batch))
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != sha256_of(source):
        return None
    if launches_per_step is not None:
        # a summary may give the traffic of several launch counts (K-chunkings):
        # traffic_bytes_per_launch@<launches per step>
        key = "traffic_bytes_per_launch@%d" % round(launches_per_step)
        if key in vals:
            try:
                return float(vals[key])
            except ValueError:
                return None
    if launches_per_step is not None and "launches_per_step" in vals:
        try:
            if abs(float(vals["launches_per_step"]) - launches_per_step) > 0.01:
                return None
        except ValueError:
            return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.gpu = gpu_index
        self.period = period_ms
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self, t0: float, t1: float):
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for (_, l) in self.lines]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --- distributed helpers (host logic; covered by gloo tests on CPU) ----------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_timing(elapsed_ms: float, units: float, device=None):
    """(max elapsed over ranks, sum of units over ranks); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_ms, units
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# --- the CPU oracle as baseline / reference arm ------------------------------

class OracleRunner:
    """The oracle's online answer on a bounded sample of one step's work: the query
    NTT of `nq` of the batch's B queries, then the fold and inverse NTT of those
    queries against `ncols` of the D2 columns, whose DB polynomials are NTT-encoded
    beforehand (as the server's DB is).  measured_s is the sample's own time;
    extrapolated_s scales the query NTT by B / nq and the fold by (B / nq)(D2 / ncols)
    to the whole answer.  With nq = B and ncols = D2 the sample is the full answer."""

    def __init__(self, n, log2p, D1, D2, B, nq, ncols, nthreads, db_seed=0, raw=None, modswitch=False):
        from oracle import oracle as O
        import synth
        self.O, self.synth = O, synth
        self.modswitch = modswitch
        self.P = O.make_params(n, log2p, D1, D2, L_PRIMES)
        self.n, self.D1, self.D2, self.B = n, D1, D2, B
        self.nq, self.ncols, self.nthreads = min(nq, B), min(ncols, D2), nthreads
        if raw is not None:
            cols = np.arange(self.ncols, dtype=np.uint64)
            ids = (np.arange(D1, dtype=np.uint64)[None, :] * np.uint64(D2) + cols[:, None]).reshape(-1)
            self.dbhat = O.encode_polys(self.P, raw, ids, nthreads)
        else:  # only the sample's polynomials, regenerated from the DB's counter-based stream
            bpp = n * log2p // 8
            compact = np.concatenate([synth.raw_db_slab(db_seed, (i * D2 + c) * bpp, bpp)
                                      for c in range(self.ncols) for i in range(D1)])
            Pc = O.make_params(n, log2p, self.ncols * D1, 1, L_PRIMES)
            self.dbhat = O.encode_polys(Pc, compact, np.arange(self.ncols * D1, dtype=np.uint64), nthreads)
        self.dbhat = self.dbhat.reshape(self.ncols, D1, L_PRIMES, n)

    @property
    def full(self):
        return self.nq == self.B and self.ncols == self.D2

    def step(self, seed):
        synth = self.synth
        Q = synth.uniform_residues(seed, synth.STREAM_UNIFORM, self.nq * self.D1 * 2, self.n, self.P.qs)
        Q = Q.reshape(self.nq, self.D1, 2, L_PRIMES, self.n)
        t0 = time.perf_counter()
        qhat = self.O.ntt_fwd_rns(self.P, Q, self.nthreads)
        t1 = time.perf_counter()
        R = self.O.answer_encoded(self.P, self.dbhat, qhat, self.nthreads)
        if self.modswitch:
            self.O.modswitch(self.P, R)
        t2 = time.perf_counter()
        scale_q = self.B / self.nq
        return {"measured_s": t2 - t0,
                "extrapolated_s": (t1 - t0) * scale_q + (t2 - t1) * scale_q * self.D2 / self.ncols}

    def describe(self):
        if self.full:
            return ("oracle online answer, full: query NTT, fold of all %d columns and inverse NTT%s for all %d "
                    "queries; the DB NTT-encoded beforehand" % (self.D2, " + modulus switching" if self.modswitch
                                                                 else "", self.B))
        return ("oracle online answer on a sample, extrapolated: query NTT of %d of %d queries, fold + inverse NTT%s "
                "of those queries on %d of %d columns (those DB columns NTT-encoded beforehand); the query NTT "
                "scaled by queries, the fold by queries x columns"
                % (self.nq, self.B, " + modulus switching" if self.modswitch else "", self.ncols, self.D2))


def oracle_sample_shape(wl, B, ref_cols):
    """(queries, columns) of the oracle's bounded sample: about a second of host work
    per step on 16 cores for the 16 GiB and 32 GiB databases, more of the batch for
    the smaller ones."""
    n, log2p, D1, D2, _, _ = WORKLOADS[wl]
    per_query = D1 * n * L_PRIMES  # grows with the work per query and column
    nq = max(1, min(B, (1 << 24) // per_query))
    return nq, max(1, min(D2, ref_cols))


def reference_arm(args, wl):
    n, log2p, D1, D2, B0, desc = WORKLOADS[wl]
    B = args.batch or B0
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import synth
    raw_bytes = synth.raw_db_bytes(n, log2p, D1, D2)
    nthreads = os.cpu_count() or 1
    nq, ncols = oracle_sample_shape(wl, B, args.ref_cols)
    runner = OracleRunner(n, log2p, D1, D2, B, nq, ncols, nthreads, db_seed=0, modswitch=args.modswitch)
    meas, extra = [], []
    for step in range(args.warmup + args.steps):
        r = runner.step(100 + step)
        if step >= args.warmup:
            meas.append(r["measured_s"])
            extra.append(r["extrapolated_s"])
    meas_s, extra_s = sum(meas) / len(meas), sum(extra) / len(extra)
    value = raw_bytes * B / extra_s / 1e9
    fraction = meas_s / extra_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": meas_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "step": ("each step runs the oracle on a bounded sample of the batch's answer (%s); ms_per_step is that "
                 "sample's measured time, value the metric over the extrapolated full answer"
                 % ("full answer" if runner.full else "%.4f of it by time" % fraction)),
        "extrapolated_ms_per_full_step": extra_s * 1e3,
        "config": {"workload": wl, "description": desc, "batch": B, "n": n, "log2p": log2p, "D1": D1, "D2": D2,
                   "L": L_PRIMES, "modswitch": bool(args.modswitch)},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": nthreads, "kind": "oracle",
                         "sample": runner.describe(), "measured_ms": meas_s * 1e3, "extrapolated_ms": extra_s * 1e3,
                         "label": "full" if runner.full else "extrapolated"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_full_answers(wl, raw, cpu_full):
    """Full oracle answers (every query, every column) on the host cores: batch 1 and
    8, on all cores and on one core.  One core at batch 8 takes minutes, so it runs
    only with cpu_full."""
    n, log2p, D1, D2, _, _ = WORKLOADS[wl]
    allc = os.cpu_count() or 1
    out = []
    runners = {}
    for B in (1, 8):
        for cores in (allc, 1):
            if B == 8 and cores == 1 and not cpu_full:
                out.append({"batch": B, "cores": cores, "skipped": "minutes of host time; bench.py --cpu-full runs it"})
                continue
            key = B
            if key not in runners:
                runners[key] = OracleRunner(n, log2p, D1, D2, B, B, D2, allc, raw=raw)
            r = runners[key]
            r.nthreads = cores
            res = r.step(300 + B)
            out.append({"batch": B, "cores": cores, "ms": res["measured_s"] * 1e3,
                        "value": synth_raw_bytes(wl) * B / res["measured_s"] / 1e9, "unit": "GB/s",
                        "label": "full"})
    return out


def synth_raw_bytes(wl):
    n, log2p, D1, D2, _, _ = WORKLOADS[wl]
    return D1 * D2 * n * log2p // 8


# --- our arm -----------------------------------------------------------------

class Ctx:
    """What every timed block of our arm shares."""

    def __init__(self, args, wl, g, binding, synth, torch, dev, rank, world, sampler):
        self.args, self.wl, self.g, self.binding, self.synth, self.torch = args, wl, g, binding, synth, torch
        self.dev, self.rank, self.world, self.sampler = dev, rank, world, sampler
        self.peaks, self.peak_kind = measured_peaks()
        self.probes = {}

    def probe(self, name, stream):
        if name not in self.probes:
            fn = {"int8": self.g.pir_probe_int8_mma}[name]
            self.probes[name] = fn(stream)
        return self.probes[name]


def gemm_roofline(ctx, layout, B, p, tile, gemm_ms, launches_per_step, clocks, stream):
    """Roofline of the dominant kernel (the modular GEMM stage) for one launch:
    the algorithmic work of one step divided by its launches, over the event-timed
    kernel time per launch.  Query rows are counted unpadded."""
    g = ctx.g
    n, D1, D2 = p.n, p.D1, p.D2
    M = 2 * B
    nslots = L_PRIMES * n
    launch_ms = gemm_ms / launches_per_step
    streaming = layout == g.PIR_LAYOUT_PLAIN and M <= 8 and (tile in (1, 2, 3, 7) or (tile == 0 and M <= 4 and D2 <= 512))
    if streaming:
        kernel_tag = "scan_tma" if tile in (0, 7) else "gemv_scan"
        alg_bytes = nslots * (D1 * D2 * 4 + D1 * M * 4 + M * D2 * 4)
        per = alg_bytes / launches_per_step
        rl = {"bound": "hbm", "achieved": per / (launch_ms / 1e3) / 1e9, "peak": float(ctx.peaks["hbm_gbs"]),
              "unit": "GB/s", "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % ctx.peak_kind}
    elif layout == g.PIR_LAYOUT_TENSOR:
        # bf16 tensor cores: 16 digit products (2 FLOP each) per modular MAC of the
        # useful query rows, against the measured sustained dense bf16 peak (the
        # kernel runs inside a long step); bytes: 8 per DB residue (four bf16 digits)
        kernel_tag = "gemm_tc"
        macs = nslots * D1 * D2 * M / launches_per_step
        alg_bytes = nslots * (D1 * D2 * 8 + D1 * M * 8 + M * D2 * 4)
        per = alg_bytes / launches_per_step
        rl = {"bound": "tensor", "achieved": 32.0 * macs / (launch_ms / 1e3) / 1e12,
              "peak": float(ctx.peaks.get("bf16_tflops_sustained", 1700.0)), "unit": "TFLOP/s",
              "peak_source": "%s bf16_tflops_sustained (MEASURED_PEAKS.json)" % ctx.peak_kind,
              "modmac_per_s": macs / (launch_ms / 1e3), "hbm_gbs": per / (launch_ms / 1e3) / 1e9,
              "hbm_frac": per / (launch_ms / 1e3) / 1e9 / float(ctx.peaks["hbm_gbs"])}
    else:
        macs = nslots * D1 * D2 * M / launches_per_step
        alg_bytes = nslots * (D1 * D2 * 4 + D1 * M * 4 + M * D2 * 4)
        per = alg_bytes / launches_per_step
        if layout == g.PIR_LAYOUT_PLAIN:
            # one mad.wide.u32 per modular MAC; that instruction holds the multiply-add
            # pipe four cycles per warp, 32 per clock per SM (the ncu pipe counters of
            # this kernel confirm it), so the peak is derived from the sampled clock
            kernel_tag = "gemm_plain"
            sm_mhz = clocks.get("sm_mhz") or float(ctx.peaks.get("sm_max_mhz", 2070.0))
            peak = 152 * 32 * sm_mhz * 1e6 / 1e12
            rl = {"bound": "alu", "achieved": macs / (launch_ms / 1e3) / 1e12, "peak": peak, "unit": "T modMAC/s",
                  "peak_source": "derived: 152 SMs x 32 mad.wide.u32 / clock x sampled SM clock %.0f MHz" % sm_mhz,
                  "hbm_gbs": per / (launch_ms / 1e3) / 1e9}
        else:
            # 16 byte products per modular MAC on the INT8 tensor pipe
            kernel_tag = "gemm_limb"
            tops = ctx.probe("int8", stream)
            rl = {"bound": "tensor", "achieved": 32.0 * macs / (launch_ms / 1e3) / 1e12, "peak": tops,
                  "unit": "TOPS (INT8 mma.sync)", "modmac_per_s": macs / (launch_ms / 1e3),
                  "peak_source": "pir_probe_int8_mma on this GPU (MEASURED_PEAKS.json has no INT8 entry)"}
    rl["frac"] = rl["achieved"] / rl["peak"]
    rl["kernel"] = kernel_tag
    rl["tile"] = tile  # the GEMM tile id the timed answers ran (0: the built-in choice)
    rl["kernel_ms"] = launch_ms
    rl["launches_per_step"] = launches_per_step
    rl["alg_bytes_per_launch"] = per
    src = os.path.join(ROOT, "paper_2606_11536_gb300", "csrc",
                       {"scan_tma": "scan_tma.cu", "gemv_scan": "gemm_plain.cu", "gemm_plain": "gemm_plain.cu",
                        "gemm_limb": "gemm_limb.cu", "gemm_tc": "gemm_tc.cu"}[kernel_tag])
    rl["traffic"] = profile_traffic(kernel_tag, ctx.wl, B, src, launches_per_step)
    return rl


def make_db(ctx, p, layout):
    """The resident DB: from host bytes up to 2 GiB raw (also what the oracle reads),
    else generated on the device from the same counter-based stream."""
    g, synth, torch = ctx.g, ctx.synth, ctx.torch
    raw_bytes = ctx.binding.raw_db_bytes(p)
    if raw_bytes <= (2 << 30):
        raw = synth.raw_db(0, raw_bytes)
        return g.pir_setup_db(p, raw, layout=layout), raw
    raw_d = synth.raw_db_torch(0, raw_bytes, device=ctx.dev)
    db = g.pir_setup_db(p, raw_d, layout=layout)
    del raw_d
    torch.cuda.empty_cache()
    return db, None


def measure_batch(ctx, db, p, layout, B, steps, warmup, min_seconds=0.0, extras=None, tuned=False):
    """Time `steps` answers of B queries (at least min_seconds of them when asked),
    after `warmup` untimed ones, with CUDA events on the launching stream, bracketed
    by barrier + synchronize.  Returns the block's numbers and its step function.

    tuned: the batching runtime's own form of a batch, as the method asks for it:
    the library's autotuner picks the GEMM tile and K-chunk for this DB and batch
    (untimed), and every timed step replays one captured graph of the answer.  The
    graph replays carry no stage events, so the dominant kernel's time for the
    roofline comes from a separate, shorter run of the same configuration with
    stage events."""
    args, g, synth, torch = ctx.args, ctx.g, ctx.synth, ctx.torch
    n, D1, D2 = p.n, p.D1, p.D2
    extras = extras or {}
    msw = g.PIR_ANSWER_MODSWITCH if args.modswitch else 0
    qwords = B * D1 * 2 * L_PRIMES * n
    rwords = B * D2 * 2 * (1 if msw else L_PRIMES) * n
    rg, ex = extras.get("rgsw"), extras.get("expander")
    if rg is not None:
        rwords = B * 2 * (1 if msw else L_PRIMES) * n
    if ex is not None:
        qwords = B * 2 * L_PRIMES * n
    # several query buffers rotate when they are small, so no step reads inputs the
    # previous step left in L2
    nbuf = 4 if qwords * 4 <= (4 << 30) else 1
    nct = qwords // (L_PRIMES * n)
    qbufs = [synth.uniform_residues_torch(1000 + 17 * ctx.rank + 5 * B + t, synth.STREAM_UNIFORM, nct, n, p.qs,
                                          device=ctx.dev).view(-1) for t in range(nbuf)]
    stream = torch.cuda.current_stream()
    nstreams = args.streams
    streams = [stream] + [torch.cuda.Stream(device=ctx.dev) for _ in range(nstreams - 1)]
    resps = [torch.empty(rwords, dtype=torch.int32, device=ctx.dev) for _ in range(nstreams)]

    tile, k_chunk = args.tile, args.k_chunk
    tuned_opts = None
    if tuned and not extras:
        tuned_opts = g.pir_autotune(db, B, stream=stream)
        tile, k_chunk = tuned_opts["tile"], tuned_opts["k_chunk"]
    graphs = None
    if args.graph or tuned_opts is not None:
        # one captured answer per query buffer, replayed (the graph binds its buffers)
        if ex is not None:
            graphs = [g.pir_graph_create_packed(db, ex, qb, B, resps[0], tile=tile, flags=msw) for qb in qbufs]
        elif rg is None:
            graphs = [g.pir_graph_create(db, qb, B, resps[0], k_chunk=k_chunk, tile=tile, flags=msw)
                      for qb in qbufs]
        else:
            raise SystemExit("--graph covers the plain and packed answers")

    def step(t, flags=0):
        st, rs = streams[t % nstreams], resps[t % nstreams]
        if graphs is not None:
            g.pir_graph_launch(graphs[t % nbuf], stream=stream)
            return
        if rg is not None:
            g.pir_answer_folded(db, qbufs[t % nbuf], B, args.ell, rg, rs, stream=st, flags=flags | msw, tile=args.tile)
        elif ex is not None:
            g.pir_answer_packed(db, ex, qbufs[t % nbuf], B, rs, stream=st, flags=flags | msw, tile=args.tile)
        elif args.noalloc:
            g.pir_answer_noalloc(db, qbufs[t % nbuf], B, rs, stream=st)
        else:
            g.pir_answer_ex(db, qbufs[t % nbuf], B, rs, stream=st, flags=flags | msw, tile=tile, k_chunk=k_chunk)

    for t in range(warmup):
        step(t)
    torch.cuda.synchronize()
    if min_seconds > 0:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(0)
        e1.record(stream)
        torch.cuda.synchronize()
        est_s = max(e0.elapsed_time(e1) / 1e3, 1e-6)
        steps = max(steps, int(np.ceil(min_seconds / est_s)))
    g.pir_stage_times()  # reset
    barrier()
    torch.cuda.synchronize()
    launches0 = g.pir_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    # an NVTX range names the timed launches for a profiler (ncu --nvtx-include)
    torch.cuda.nvtx.range_push("timed_b%d_%s" % (B, {g.PIR_LAYOUT_PLAIN: "plain", g.PIR_LAYOUT_LIMB: "limb",
                                                    g.PIR_LAYOUT_TENSOR: "tensor"}[layout]))
    ev0.record(stream)
    for st in streams[1:]:
        st.wait_event(ev0)
    for t in range(steps):
        step(t, flags=g.PIR_ANSWER_STAGE_TIMES)
    for st in streams[1:]:
        stream.wait_stream(st)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    w1 = time.time()
    barrier()
    launches = g.pir_kernel_launches() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    stage_ms, stage_launches = g.pir_stage_times()
    clocks = ctx.sampler.summary(w0, w1)
    max_ms, total_queries = reduce_timing(elapsed_ms, float(B * steps), device=ctx.dev if ctx.world > 1 else None)
    raw_bytes = ctx.binding.raw_db_bytes(p)
    rl_steps, rl_note = steps, "stage events of the timed steps"
    if graphs is not None and ex is None:
        # the graph replays carry no stage events: time the same configuration with
        # them, outside the graph, for the dominant kernel's duration
        rl_steps = max(3, int(np.ceil(0.5 / max(max_ms / steps / 1e3, 1e-6))))
        g.pir_stage_times()
        for t in range(rl_steps):
            g.pir_answer_ex(db, qbufs[t % nbuf], B, resps[0], stream=stream, flags=g.PIR_ANSWER_STAGE_TIMES | msw,
                            tile=tile, k_chunk=k_chunk)
        torch.cuda.synchronize()
        stage_ms, stage_launches = g.pir_stage_times()
        rl_note = ("stage events of %d answers of the same configuration outside the graph (the replays carry "
                   "none)" % rl_steps)
    gemm_launches = max(1, stage_launches[2])
    launches_per_step = gemm_launches / rl_steps
    gemm_ms = stage_ms[2] / rl_steps  # GEMM kernel time per step
    if stage_launches[2] == 0:  # an entry point without stage events: the whole step bounds the GEMM
        gemm_ms, launches_per_step = max_ms / steps, 1.0
    roofline = gemm_roofline(ctx, layout, B, p, tile, gemm_ms, launches_per_step, clocks, stream)
    roofline["stage_ms_per_step"] = {name: stage_ms[i] / rl_steps for i, name in enumerate(ctx.binding.STAGE_NAMES)}
    roofline["kernel_timed_with"] = rl_note
    for gr in graphs or []:
        g.pir_graph_destroy(gr)
    out = {"batch": B, "value": raw_bytes * total_queries / (max_ms / 1e3) / 1e9, "unit": "GB/s",
           "ms_per_step": max_ms / steps, "steps": steps, "warmup": warmup, "timed_s": max_ms / 1e3,
           "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks,
           "launch": ("one captured graph per batch, autotuned tile %d, K-chunk %d" % (tile, k_chunk)
                      if tuned_opts is not None else "graph replay" if graphs is not None else "pir_answer_ex")}
    return out, {"qbufs": qbufs, "qwords": qwords, "rwords": rwords, "stream": stream, "msw": msw}


def measure_e2e(ctx, db, p, B, bufs, extras, est_step_ms):
    """The same metric through the public API with pinned host buffers: every step
    copies its queries host -> device and its responses back inside the call."""
    args, g, torch = ctx.args, ctx.g, ctx.torch
    qwords, rwords, stream, msw = bufs["qwords"], bufs["rwords"], bufs["stream"], bufs["msw"]
    rg, ex = extras.get("rgsw"), extras.get("expander")
    try:
        host_ram = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        host_ram = 64 << 30
    if (qwords + rwords) * 4 > host_ram // 2:
        return None
    qh = torch.empty(qwords, dtype=torch.int32, pin_memory=True)
    rh = torch.empty(rwords, dtype=torch.int32, pin_memory=True)
    qh.copy_(bufs["qbufs"][0])
    rgh = None
    if rg is not None:
        rgh = torch.empty(rg.numel(), dtype=torch.int32, pin_memory=True)
        rgh.copy_(rg.cpu())
    n_steps = max(3, min(args.steps, int(np.ceil(1000.0 / max(est_step_ms, 1e-3)))))

    def e2e_step():
        if rg is not None:
            g.pir_answer_folded(db, qh, B, args.ell, rgh, rh, stream=stream, flags=msw)
        elif ex is not None:
            g.pir_answer_packed(db, ex, qh, B, rh, stream=stream, flags=msw)
        else:
            g.pir_answer_ex(db, qh, B, rh, stream=stream, flags=msw)
    for _ in range(2):
        e2e_step()
    barrier()
    step_ms = []
    t0 = time.perf_counter()
    for _ in range(n_steps):
        e2e_step()
        step_ms.append((time.perf_counter() - t0) * 1e3 - sum(step_ms))
    t1 = time.perf_counter()
    e2e_ms, e2e_q = reduce_timing((t1 - t0) * 1e3, float(B * n_steps), device=ctx.dev if ctx.world > 1 else None)
    raw_bytes = ctx.binding.raw_db_bytes(p)
    return {"value": raw_bytes * e2e_q / (e2e_ms / 1e3) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": qwords * 4 + (rg.numel() * 4 if rg is not None else 0),
            "d2h_bytes_per_step": rwords * 4, "ms_per_step": e2e_ms / n_steps, "steps": n_steps,
            "step_ms_min": min(step_ms), "step_ms_max": max(step_ms), "step_ms": [round(t, 2) for t in step_ms]}


def our_arm(args, wl):
    import torch
    import paper_2606_11536_gb300 as g
    from paper_2606_11536_gb300 import binding
    import synth

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                           else int(os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local]))
    sampler.start()
    ctx = Ctx(args, wl, g, binding, synth, torch, dev, rank, world, sampler)

    n, log2p, D1, D2, B0, desc = WORKLOADS[wl]
    B = args.batch or B0
    layout = {"plain": g.PIR_LAYOUT_PLAIN, "limb": g.PIR_LAYOUT_LIMB, "tensor": g.PIR_LAYOUT_TENSOR}[args.layout]
    p = g.pir_make_params(n, log2p, D1, D2, L_PRIMES)
    raw_bytes = binding.raw_db_bytes(p)
    db, raw = make_db(ctx, p, layout)

    if args.packed and args.folded:
        raise SystemExit("--packed and --folded are separate modes")
    extras = {}
    if args.folded:
        # RGSW rows of the log2(D2) remaining levels per query; the external products'
        # cost does not depend on their values, so timing-only rows are uniform residues
        flevels = max(0, (D2 - 1).bit_length())
        extras["rgsw"] = synth.uniform_residues_torch(78, synth.STREAM_KEY_A, B * flevels * 2 * args.ell * 2, n,
                                                      p.qs, device=dev).view(-1)
    if args.packed:
        # packed queries (one ciphertext each) expanded on the GPU; the expansion's
        # cost does not depend on the key values, so timing-only keys are uniform
        # residues of the key shape [levels][ell][2][L][n]
        levels = max(0, (D1 - 1).bit_length())
        keys = synth.uniform_residues_torch(77, synth.STREAM_KEY_A, levels * args.ell * 2, n, p.qs, device=dev)
        extras["expander"] = g.pir_expander_create(p, levels, args.ell, keys.view(-1))
        del keys

    time.sleep(0.3)  # clock samples before the first timed region
    # the default line answers each batch the way the batching runtime does: the
    # autotuner's tile and K-chunk, one captured graph per batch (--untuned: the
    # built-in choice through pir_answer_ex)
    tuned = not args.untuned and not args.graph and not extras and args.tile == 0 and args.k_chunk == 0 and \
        args.streams == 1 and not args.noalloc
    head, bufs = measure_batch(ctx, db, p, layout, B, args.steps, args.warmup, extras=extras, tuned=tuned)
    e2e = measure_e2e(ctx, db, p, B, bufs, extras, head["ms_per_step"])
    del bufs

    # the metric's batch range and the tensor layout, on the default workload (one GPU)
    plain_mode = layout == g.PIR_LAYOUT_PLAIN and not extras and args.streams == 1 and args.tile == 0 and \
        args.k_chunk == 0 and not args.modswitch and not args.noalloc and not args.graph and wl == DEFAULT_WORKLOAD
    per_batch = tensor_block = None
    if world == 1 and plain_mode and args.per_batch:
        per_batch = []
        for b in PER_BATCH:
            if b == B:
                r = {k: head[k] for k in ("batch", "value", "unit", "ms_per_step", "steps", "warmup", "timed_s",
                                          "roofline", "gpu_launches", "clocks", "launch")}
                r["headline"] = True
            else:
                r = measure_batch(ctx, db, p, layout, b, 3, 3, min_seconds=MIN_TIMED_S, tuned=tuned)[0]
                torch.cuda.empty_cache()
            per_batch.append(r)
    if world == 1 and plain_mode and args.tensor_block:
        g.pir_free_db(db)
        db = None
        torch.cuda.empty_cache()
        tdb, _ = make_db(ctx, p, g.PIR_LAYOUT_TENSOR)
        try:
            tb = 32 if B != 32 and not args.batch else B
            r = measure_batch(ctx, tdb, p, g.PIR_LAYOUT_TENSOR, tb, 3, 3, min_seconds=MIN_TIMED_S, tuned=tuned)[0]
        finally:
            g.pir_free_db(tdb)
            torch.cuda.empty_cache()
        plain_ref = next((x for x in (per_batch or []) if x["batch"] == tb), head if tb == B else None)
        r["layout"] = "tensor (opt-in: bf16 tcgen05 digits, 8 bytes per residue, exact integer results)"
        r["resident_bytes"] = binding.resident_db_bytes(p, g.PIR_LAYOUT_TENSOR)
        if plain_ref is not None:
            pg = plain_ref["roofline"]["stage_ms_per_step"]["gemm"]
            tg = r["roofline"]["stage_ms_per_step"]["gemm"]
            r["gemm_ms_plain"], r["gemm_ms_tensor"] = pg, tg
            r["gemm_speedup_vs_plain"] = pg / tg
            r["step_speedup_vs_plain"] = plain_ref["ms_per_step"] / r["ms_per_step"]
        tensor_block = r

    # the largest single-GPU configuration (32 GiB raw, 128 GiB resident) at batch 64
    # on the plain path and on the exact limb-INT8 tensor path (the benchmark spec's
    # comparison), each timed for at least a second
    large = None
    if world == 1 and plain_mode and args.large_block:
        if db is not None:
            g.pir_free_db(db)
            db = None
            torch.cuda.empty_cache()
        wl5 = "db32g_n8192"
        n5, lp5, D15, D25, B5, desc5 = WORKLOADS[wl5]
        p5 = g.pir_make_params(n5, lp5, D15, D25, L_PRIMES)
        large = {"workload": wl5, "description": desc5, "batch": B5}
        ctx.wl = wl5
        for name, lay in (("plain", g.PIR_LAYOUT_PLAIN), ("limb", g.PIR_LAYOUT_LIMB)):
            db5, _ = make_db(ctx, p5, lay)
            try:
                r = measure_batch(ctx, db5, p5, lay, B5, 2, 3, min_seconds=MIN_TIMED_S)[0]
            finally:
                g.pir_free_db(db5)
                torch.cuda.empty_cache()
            large[name] = r
        ctx.wl = wl
        large["limb_vs_plain"] = large["plain"]["ms_per_step"] / large["limb"]["ms_per_step"]

    # the metric's serving half: the serving configuration at one offered load
    serving_blk = None
    if world == 1 and plain_mode and args.serving_block:
        if db is not None:
            g.pir_free_db(db)
            db = None
        torch.cuda.empty_cache()
        g.pir_release_memory()
        # a child process, as `bench.py --serving` runs: its allocators start empty, so
        # the 208 GiB of resident serving DBs meet no cache left by the blocks above.
        # Uncaptured dispatch: with captured graphs an overloaded sweep has stalled
        # (two batches that never completed), without them it has not
        cmd = [sys.executable, os.path.abspath(__file__), "--serving",
               "--serving-rates", str(args.serving_block_rate), "--serving-seconds", str(args.serving_block_seconds),
               "--serving-warmup", "1.5"]
        serving_blk = serving_block_from_child(cmd, timeout_s=300)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not (args.packed or args.folded):
        nthreads = os.cpu_count() or 1
        nq, ncols = oracle_sample_shape(wl, B, args.ref_cols)
        runner = OracleRunner(n, log2p, D1, D2, B, nq, ncols, nthreads, db_seed=0, raw=raw,
                              modswitch=args.modswitch)
        runner.step(7)  # warm
        rs = [runner.step(8), runner.step(9)]
        best = min(rs, key=lambda r: r["extrapolated_s"])
        cpu = {"value": raw_bytes * B / best["extrapolated_s"] / 1e9, "unit": "GB/s", "cores": nthreads,
               "kind": "oracle", "sample": runner.describe() + "; best of 2 steps",
               "measured_ms": best["measured_s"] * 1e3, "extrapolated_ms": best["extrapolated_s"] * 1e3,
               "label": "full" if runner.full else "extrapolated"}
        if raw is not None and wl == "db1g_n4096":
            cpu["full_answers"] = oracle_full_answers(wl, raw, args.cpu_full)

    for k in ("expander",):
        if k in extras:
            g.pir_expander_free(extras[k])
    if db is not None:
        g.pir_free_db(db)
    sampler.stop()
    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": "GB/s", "n_gpus": world, "steps": head["steps"],
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wl, "description": desc, "batch": B, "n": n, "log2p": log2p, "D1": D1, "D2": D2,
                       "L": L_PRIMES, "layout": args.layout, "modswitch": bool(args.modswitch),
                       "streams": args.streams,
                       "responses": ("folded to one ciphertext per query by %d RGSW external-product levels "
                                     "(%d gadget digits; timing-only RGSW rows)" % ((D2 - 1).bit_length(), args.ell)
                                     if args.folded else "D2 ciphertexts each"),
                       "queries": ("packed, expanded on the GPU (levels %d, %d gadget digits; timing-only keys)"
                                   % ((D1 - 1).bit_length(), args.ell) if args.packed else "D1 ciphertexts each"),
                       "entry": ("pir_answer_noalloc" if args.noalloc else "pir_graph_launch" if args.graph
                                 else "pir_autotune + pir_graph_launch" if tuned else "pir_answer_ex"),
                       "launch": head["launch"],
                       "parallelism": "replicas x%d" % world,
                       "l2": "inputs larger than L2: the %.1f GiB NTT-form DB is streamed every step; query "
                             "buffers rotate when small" % (binding.resident_db_bytes(p, layout) / 2 ** 30)},
            "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": head["gpu_launches"],
            "clocks": head["clocks"], "timed_s": head["timed_s"],
        }
        if per_batch is not None:
            line["per_batch"] = per_batch
        if tensor_block is not None:
            line["tensor_layout"] = tensor_block
        if large is not None:
            line["largest_config"] = large
        if serving_blk is not None:
            line["serving"] = serving_blk
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tensor_large_bench(args):
    """The 32 GiB database (n = 8192, 8192 x 256) in the tensor layout: 256 GiB
    resident (8 bytes per residue), so a batch's queries (64 GiB at batch 64) cannot
    sit beside it on the device.  They stay in pinned host memory and each answer is
    the streamed host-buffer call (1 GiB pieces along D1, uploads behind the scan):
    the line measures that end-to-end call.  The raw DB goes up chunk by chunk from
    pinned host memory as well."""
    import torch
    import paper_2606_11536_gb300 as g
    from paper_2606_11536_gb300 import binding
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = "db32g_n8192"
    n, log2p, D1, D2, B0, desc = WORKLOADS[wl]
    B = args.batch or B0
    p = g.pir_make_params(n, log2p, D1, D2, L_PRIMES)
    raw_bytes = binding.raw_db_bytes(p)
    qwords, rwords = B * D1 * 2 * L_PRIMES * n, B * D2 * 2 * L_PRIMES * n
    # host inputs, generated on the device (same counter-based streams) and copied out
    qh = torch.empty(qwords, dtype=torch.int32, pin_memory=True)
    per = max(1, (4 << 30) // (D1 * 2 * L_PRIMES * n * 4))  # queries per 4 GiB piece
    for b0 in range(0, B, per):
        nb = min(per, B - b0)
        piece = synth.uniform_residues_torch(1000, synth.STREAM_UNIFORM, nb * D1 * 2, n, p.qs, device=dev,
                                             start=b0 * D1 * 2).view(-1)
        qh[b0 * D1 * 2 * L_PRIMES * n:(b0 + nb) * D1 * 2 * L_PRIMES * n].copy_(piece)
        del piece
    rawh = torch.empty(raw_bytes, dtype=torch.uint8, pin_memory=True)
    rawh.copy_(synth.raw_db_torch(0, raw_bytes, device=dev))
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    db = g.pir_setup_db(p, rawh, layout=g.PIR_LAYOUT_TENSOR)
    setup_s = time.perf_counter() - t0
    del rawh
    rh = torch.empty(rwords, dtype=torch.int32, pin_memory=True)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    for _ in range(args.warmup):
        g.pir_answer_ex(db, qh, B, rh, stream=stream)
    g.pir_stage_times()
    launches0 = g.pir_kernel_launches()
    w0 = time.time()
    torch.cuda.nvtx.range_push("timed_b%d_tensor_host" % B)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.pir_answer_ex(db, qh, B, rh, stream=stream, flags=g.PIR_ANSWER_STAGE_TIMES)
    ms = (time.perf_counter() - t0) * 1e3 / args.steps
    torch.cuda.nvtx.range_pop()
    w1 = time.time()
    launches = g.pir_kernel_launches() - launches0
    stage_ms, stage_launches = g.pir_stage_times()
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    g.pir_free_db(db)
    gemm_ms = stage_ms[2] / args.steps
    macs = L_PRIMES * n * D1 * D2 * 2 * B
    peaks, kind = measured_peaks()
    tflops = 32.0 * macs / (gemm_ms / 1e3) / 1e12
    value = raw_bytes * B / (ms / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": wl, "description": desc, "batch": B, "layout": "tensor",
                       "resident_bytes": binding.resident_db_bytes(p, g.PIR_LAYOUT_TENSOR), "setup_s": setup_s,
                       "timed": "end to end: each step uploads its 64 GiB of queries from pinned host memory in 1 GiB "
                                "pieces (the streamed answer) and downloads the responses; the queries cannot stay "
                                "on the device beside the 256 GiB resident DB"},
            "roofline": {"bound": "tensor", "kernel": "gemm_tc", "achieved": tflops,
                         "peak": float(peaks.get("bf16_tflops_sustained", 1700.0)), "unit": "TFLOP/s",
                         "frac": tflops / float(peaks.get("bf16_tflops_sustained", 1700.0)),
                         "gemm_ms_per_step": gemm_ms, "launches_per_step": stage_launches[2] / args.steps,
                         "stage_ms_per_step": {nm: stage_ms[i] / args.steps for i, nm in enumerate(binding.STAGE_NAMES)},
                         "traffic": None},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": qwords * 4, "d2h_bytes_per_step": rwords * 4},
            "gpu_launches": int(launches), "clocks": clocks}
    print(json.dumps(line), flush=True)


def ntt_sweep(args):
    """Standalone NTT sweep: forward then inverse NTT (in place) of 2^16 RNS
    polynomials (L = 2, n = 4096, 2 GiB) per step."""
    import torch
    import paper_2606_11536_gb300 as g
    import synth
    torch.cuda.set_device(0)
    n, count = 4096, 1 << 16
    p = g.pir_make_params(n, 16, 1, 1, L_PRIMES)
    a = synth.uniform_residues_torch(3, synth.STREAM_UNIFORM, count, n, p.qs, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        g.ntt_fwd(p, a, stream=stream)
        g.ntt_inv(p, a, stream=stream)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fwd_ms = inv_ms = 0.0
    for _ in range(args.steps):
        e0.record(stream)
        g.ntt_fwd(p, a, stream=stream)
        e1.record(stream)
        g.ntt_inv(p, a, stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        fwd_ms += e0.elapsed_time(e1)
        inv_ms += e1.elapsed_time(e2)
    nbytes = count * L_PRIMES * n * 4
    peaks, kind = measured_peaks()
    fwd_gbs = 2 * nbytes / (fwd_ms / args.steps / 1e3) / 1e9
    inv_gbs = 2 * nbytes / (inv_ms / args.steps / 1e3) / 1e9
    line = {"metric": "NTT sweep GB/s (bytes read + written per transform)", "value": fwd_gbs, "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "ntt_sweep_n4096", "polys": count, "n": n, "L": L_PRIMES, "bytes": nbytes},
            "forward_ms": fwd_ms / args.steps, "inverse_ms": inv_ms / args.steps, "inverse_gbs": inv_gbs,
            "butterflies_per_s": count * L_PRIMES * (n // 2) * 12 / (fwd_ms / args.steps / 1e3),
            "roofline": {"bound": "hbm", "achieved": fwd_gbs, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                         "frac": fwd_gbs / float(peaks["hbm_gbs"]), "peak_source": kind}}
    print(json.dumps(line), flush=True)


LWE_WORKLOADS = {  # name: (D1, D0, description); the raw INT8 DB is the operand
    "lwe1g": (1 << 15, 1 << 15, "1 GiB INT8 DB, 32768 x 32768"),
    "lwe16g": (1 << 17, 1 << 17, "16 GiB INT8 DB, 131072 x 131072"),
    "lwe64g": (1 << 18, 1 << 18, "64 GiB INT8 DB, 262144 x 262144"),
}


def lwe_bench(args):
    """Scalar-HE (LWE) DB GEMM of SimplePIR's online step: out = DB Q^T mod 2^32 on
    the raw INT8 DB (Sec. 2.5, 4.1), B queries per step."""
    import torch
    import paper_2606_11536_gb300 as g
    import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    D1, D0, desc = LWE_WORKLOADS[args.lwe_workload]
    B = args.batch or 32
    path = {"auto": g.PIR_LWE_AUTO, "tensor": g.PIR_LWE_TENSOR, "simt": g.PIR_LWE_SIMT}[args.lwe_path]
    if path == g.PIR_LWE_AUTO:
        path = g.PIR_LWE_TENSOR if B >= 8 else g.PIR_LWE_SIMT
    db = synth.raw_db_torch(0, D1 * D0, device=dev).view(torch.int8)  # uniform INT8 plaintexts
    nbuf = 2
    # query entries: uniform Z_2^32 words (both halves of each counter-based u64 draw)
    qs = [synth.u64_torch(40 + t, synth.STREAM_UNIFORM, 0, (B * D0 + 1) // 2, device=dev).view(torch.int32)[:B * D0]
          .contiguous() for t in range(nbuf)]
    out = torch.empty(B * D1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    peak_tops = g.pir_probe_int8_mma(stream)

    def step(t):
        g.pir_lwe_answer(db, D1, D0, qs[t % nbuf], B, out, path=path, stream=stream)

    for t in range(args.warmup):
        step(t)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    launches0 = g.pir_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    e0.record(stream)
    for t in range(args.steps):
        step(t)
    e1.record(stream)
    torch.cuda.synchronize()
    w1 = time.time()
    launches = g.pir_kernel_launches() - launches0
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    ms = e0.elapsed_time(e1) / args.steps
    raw = D1 * D0
    value = raw * B / (ms / 1e3) / 1e9
    macs = D1 * D0 * B
    peaks, kind = measured_peaks()
    if path == g.PIR_LWE_TENSOR:
        achieved = 2.0 * 4 * macs / (ms / 1e3) / 1e12  # four byte planes per INT8 x INT32 product
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_tops, "unit": "TOPS (INT8 mma.sync)",
                    "frac": achieved / peak_tops, "traffic": None, "kernel": "lwe_mma",
                    "peak_source": "pir_probe_int8_mma on this GPU (MEASURED_PEAKS.json has no INT8 entry)",
                    "hbm_frac": (raw * -(-B // (16 if B >= 16 else 8)) / (ms / 1e3) / 1e9) / float(peaks["hbm_gbs"])}
    else:
        achieved = raw * -(-B // min(B, 4)) / (ms / 1e3) / 1e9  # the DB streams once per group of 4 queries
        roofline = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                    "frac": achieved / float(peaks["hbm_gbs"]), "traffic": None, "kernel": "lwe_dp4a",
                    "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % kind}
    # end to end: queries from pinned host memory, results back to the host
    qh = torch.empty(B * D0, dtype=torch.int32, pin_memory=True)
    oh = torch.empty(B * D1, dtype=torch.int32, pin_memory=True)
    qh.copy_(qs[0].cpu())
    qd = torch.empty_like(qs[0])

    def e2e_step():
        qd.copy_(qh, non_blocking=True)
        g.pir_lwe_answer(db, D1, D0, qd, B, out, path=path, stream=stream)
        oh.copy_(out, non_blocking=True)
        stream.synchronize()

    e2e_step()
    t0 = time.perf_counter()
    n_e2e = max(3, min(args.steps, 20))
    for _ in range(n_e2e):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        rows = 64
        A = synth.raw_db(0, rows * D0).view(np.int8).reshape(rows, D0)  # the DB's first rows
        Qh = qh.numpy().view(np.uint32).reshape(B, D0)
        t0 = time.perf_counter()
        O.lwe_gemm(A, Qh)
        cs = time.perf_counter() - t0
        cpu = {"value": rows * D0 * B / cs / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "oracle GEMM of the first %d DB rows x %d queries, one core" % (rows, B)}
    line = {"metric": "scalar-HE DB GEMM GB/s (raw INT8 DB bytes x queries/s)", "value": value, "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "s8 x u32 mod 2^32", "data": "synthetic",
            "config": {"workload": args.lwe_workload, "description": desc, "D1": D1, "D0": D0, "batch": B,
                       "path": "tensor" if path == g.PIR_LWE_TENSOR else "dp4a",
                       "l2": "inputs larger than L2: the %.0f GiB DB streams every step" % (raw / 2 ** 30)},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": raw * B / (e2e_ms / 1e3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": B * D0 * 4,
                    "d2h_bytes_per_step": B * D1 * 4, "ms_per_step": e2e_ms},
            "gpu_launches": int(launches), "clocks": clocks, "modmac_per_s": macs / (ms / 1e3)}
    print(json.dumps(line), flush=True)


SERVING_DBS = [  # name, n, log2p, D1, D2
    ("db1g_n2048", 2048, 16, 512, 512),
    ("db1g_n4096", 4096, 16, 512, 256),
    ("db16g_n4096", 4096, 16, 4096, 512),
]
SERVING_EXTRA = ("db8g_n4096", 4096, 16, 2048, 512)


def run_serving(args, rates, seconds, graphs, warmup_s=0.0, emit=None):
    """Serving: three resident DBs, admission of a fourth by free-HBM check, Poisson
    arrivals at each offered load in `rates` for `seconds` each, uniformly random
    target DB, continuous batching.  The DBs' raw bytes are generated on the device
    from the same counter-based streams as the host generator's.  Returns the JSON
    line (p99 of the headline load as its value) and frees the DBs; emit(line), if
    given, gets the line before the DBs are freed (freeing waits for the device).
    A load in which batches ran out of time ends the sweep: the device may be
    stuck, so nothing after it waits on the device."""
    import torch
    import paper_2606_11536_gb300 as g
    from paper_2606_11536_gb300 import serving
    import synth
    serving_layout = {"plain": g.PIR_LAYOUT_PLAIN, "tensor": g.PIR_LAYOUT_TENSOR}[args.serving_layout]
    be = serving.CudaBackend(graphs=graphs, max_batch=args.serving_max_batch,
                             graph_budget=args.serving_graph_gib << 30)
    big = SERVING_DBS[-1][0]  # the 16 GiB database: its long batches may hold only some of the slots
    srv = serving.Server(be, streams=args.serving_streams, max_batch=args.serving_max_batch,
                         scratch_budget=args.serving_scratch_gib << 30, batch_timeout=args.serving_timeout,
                         db_max_slots={big: args.serving_big_slots} if args.serving_big_slots else None)
    pools = {}
    t0 = time.perf_counter()
    def device_raw(seed, n, log2p, D1, D2):
        return synth.raw_db_torch(seed, synth.raw_db_bytes(n, log2p, D1, D2), device="cuda")

    for k, (name, n, log2p, D1, D2) in enumerate(SERVING_DBS):
        p = g.pir_make_params(n, log2p, D1, D2, L_PRIMES)
        raw = device_raw(k, n, log2p, D1, D2)
        srv.admit(name, p, raw, layout=serving_layout)
        del raw
        pools[name] = [synth.uniform_residues_torch(900 + 16 * k + t, synth.STREAM_UNIFORM, D1 * 2, n, p.qs,
                                                    device="cuda").view(-1) for t in range(4)]
    name, n, log2p, D1, D2 = SERVING_EXTRA
    p = g.pir_make_params(n, log2p, D1, D2, L_PRIMES)
    torch.cuda.empty_cache()
    raw = device_raw(7, n, log2p, D1, D2)
    free_before = torch.cuda.mem_get_info()[0]
    try:
        srv.admit(name, p, raw, layout=serving_layout)
        admitted = True
    except serving.AdmissionError as e:
        admitted, err = False, str(e)
    del raw
    torch.cuda.empty_cache()
    setup_s = time.perf_counter() - t0
    dbs = list(srv.dbs)
    if admitted:
        pools[name] = [synth.uniform_residues_torch(990 + t, synth.STREAM_UNIFORM, D1 * 2, n, p.qs,
                                                    device="cuda").view(-1) for t in range(4)]
    prewarm_s = 0.0
    if graphs:
        t1 = time.perf_counter()
        be.prewarm(srv)
        prewarm_s = time.perf_counter() - t1
    if warmup_s > 0:
        # an unreported load first: the allocators' caches and the tuned tiles are
        # in place before the measured loads, as in a server that has been running
        arr = serving.poisson_arrivals(rates[0], warmup_s, dbs, seed=7,
                                       make_query=lambda db, k: pools[db][k % len(pools[db])])
        if not any(r.status == serving.PIR_ERR_TIMEOUT for r in srv.run(arr)):
            torch.cuda.synchronize()
    results = []
    stopped = None
    for rate in rates:
        arr = serving.poisson_arrivals(rate, seconds, dbs, seed=int(rate),
                                       make_query=lambda db, k: pools[db][k % len(pools[db])])
        done = srv.run(arr)
        st = serving.latency_stats(done)
        st["offered_qps"] = rate
        st["saturated"] = st.get("qps", 0.0) < 0.9 * rate
        st["per_db"] = {d: serving.latency_stats([r for r in done if r.db == d]) for d in dbs}
        results.append(st)
        if any(r.status == serving.PIR_ERR_TIMEOUT for r in done):
            stopped = "batches ran out of time at %g q/s; later loads not run" % rate
            break
        torch.cuda.synchronize()  # the next load starts on an idle device
    try:
        g.pir_device_status()  # a bounded kernel wait that ran out (reads without waiting)
        device_status = 0
    except g.PirError as e:
        device_status = e.status
    # the headline: p99 at the stated load (the highest offered rate the server kept up with
    # unless one is named)
    if args.serving_headline_rate:
        head = next(r for r in results if r["offered_qps"] == args.serving_headline_rate)
    else:
        kept = [r for r in results if not r["saturated"]]
        head = max(kept, key=lambda r: r["offered_qps"]) if kept else results[0]
    line = {"metric": "serving p50/p99 ms (Poisson arrivals, continuous batching)", "unit": "ms",
            "value": head.get("p99_ms"), "p50_ms": head.get("p50_ms"), "achieved_qps": head.get("qps"),
            "offered_qps": head["offered_qps"], "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": "u32",
            "config": {"workload": "serving", "dbs": [d[0] for d in SERVING_DBS], "fourth_db": SERVING_EXTRA[0],
                       "fourth_admitted": admitted, "free_hbm_before_fourth": free_before,
                       "streams": args.serving_streams, "max_batch": args.serving_max_batch,
                       "layout": args.serving_layout, "graphs": bool(graphs),
                       "big_db_slot_cap": args.serving_big_slots, "batch_timeout_s": args.serving_timeout,
                       "seconds_per_load": seconds, "warmup_load_s": warmup_s, "setup_s": setup_s,
                       "graph_prewarm_s": prewarm_s,
                       "resident_bytes": srv.resident_bytes},
            "graph_launches": be.graph_launches, "failed": len(srv.failed), "device_status": device_status,
            "loads": results}
    if stopped:
        line["stopped"] = stopped
    if emit is not None:
        emit(line)
    if not stopped:  # (after a stopped sweep a batch may still hold its DB: the process ends as is)
        for d in list(srv.dbs):  # frees each DB and the graphs made for it
            srv.evict(d)
        torch.cuda.empty_cache()
    return line


def serving_block_from_child(cmd, timeout_s):
    """Runs the serving benchmark `cmd` in a child process and returns the default
    line's `serving` block from the JSON line it prints.  The child prints its line
    before it frees its databases (which waits for the device): if it then runs past
    timeout_s, the line is kept with a note.  Anything else that goes wrong is
    recorded in the block as an error; the caller's line stands without it."""
    metric = "serving p50/p99 ms (Poisson arrivals, continuous batching)"
    note = None
    try:
        try:
            child = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
            out = child.stdout
            if child.returncode != 0:
                if not (out or "").strip():
                    raise RuntimeError("exit %d: %s" % (child.returncode, (child.stderr or "")[-600:]))
                note = "the serving process exited with %d after printing its line" % child.returncode
        except subprocess.TimeoutExpired as e:
            out = e.stdout.decode() if isinstance(e.stdout, bytes) else (e.stdout or "")
            if not out.strip():
                raise
            note = "the serving process did not end within %d s after its loads" % timeout_s
        sl = json.loads(out.strip().splitlines()[-1])
        ld = sl["loads"][0]
        blk = {"metric": sl.get("metric", metric), "unit": "ms", "p50_ms": ld.get("p50_ms"),
               "p99_ms": ld.get("p99_ms"), "offered_qps": ld["offered_qps"], "achieved_qps": ld.get("qps"),
               "saturated": ld.get("saturated"), "mean_batch": ld.get("mean_batch"), "failed": sl.get("failed"),
               "graph_launches": sl.get("graph_launches"), "config": sl.get("config"),
               "device_status": sl.get("device_status"),
               "per_db_p99_ms": {d: v.get("p99_ms") for d, v in ld.get("per_db", {}).items()}}
        if sl.get("stopped"):
            blk["stopped"] = sl["stopped"]
        if note:
            blk["note"] = note
        return blk
    except Exception as e:  # the block is optional: record why it is missing
        return {"metric": metric, "error": "%s: %s" % (type(e).__name__, str(e)[:600])}


def serving_bench(args):
    import torch
    torch.cuda.set_device(0)
    run_serving(args, args.serving_rates, args.serving_seconds, args.serving_graphs, warmup_s=args.serving_warmup,
                emit=lambda line: print(json.dumps(line), flush=True))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--layout", default="plain", choices=["plain", "limb", "tensor"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=0, help="GEMM tile id (0 = built-in choice)")
    ap.add_argument("--k-chunk", type=int, default=0, help="fold D1 in chunks of this many ciphertexts")
    ap.add_argument("--ref-cols", type=int, default=16, help="columns in the oracle's timed sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="with --workload db1g_n4096: also the full oracle answer of batch 8 on one core (minutes)")
    ap.add_argument("--no-per-batch", dest="per_batch", action="store_false",
                    help="skip the per-batch blocks (batches 1, 8, 32, 128) of the default plain run")
    ap.add_argument("--no-tensor-block", dest="tensor_block", action="store_false",
                    help="skip the tensor-layout block (batch 32) of the default plain run")
    ap.add_argument("--no-large-block", dest="large_block", action="store_false",
                    help="skip the 32 GiB block (batch 64, plain and limb layouts) of the default plain run")
    ap.add_argument("--lwe", action="store_true", help="time the scalar-HE (LWE) INT8 x INT32 DB GEMM instead")
    ap.add_argument("--lwe-workload", default="lwe16g", choices=sorted(LWE_WORKLOADS))
    ap.add_argument("--lwe-path", default="auto", choices=["auto", "tensor", "simt"])
    ap.add_argument("--packed", action="store_true",
                    help="one packed ciphertext per query, expanded on the GPU (pir_answer_packed)")
    ap.add_argument("--streams", type=int, default=1,
                    help="CUDA streams the steps go round-robin over (answers in flight at once)")
    ap.add_argument("--folded", action="store_true",
                    help="fold the D2 responses into one per query with RGSW external products (pir_answer_folded)")
    ap.add_argument("--ell", type=int, default=4, help="gadget digits of the expansion keys / RGSW rows")
    ap.add_argument("--modswitch", action="store_true",
                    help="switch the responses to the single prime q_0 inside the inverse NTT")
    ap.add_argument("--ntt-sweep", action="store_true", help="time the standalone NTT sweep instead")
    ap.add_argument("--tensor-large", action="store_true",
                    help="the 32 GiB DB in the tensor layout (256 GiB resident), answered from pinned host queries")
    ap.add_argument("--untuned", action="store_true",
                    help="time the built-in tile / K-chunk choice through pir_answer_ex (no autotuner, no graphs)")
    ap.add_argument("--graph", action="store_true",
                    help="replay captured answers (pir_graph_create, pir_graph_create_packed with --packed)")
    ap.add_argument("--noalloc", action="store_true",
                    help="answer through pir_answer_noalloc (the library's fixed scratch array, no allocation)")
    ap.add_argument("--serving", action="store_true", help="run the serving benchmark instead")
    ap.add_argument("--no-serving-block", dest="serving_block", action="store_false",
                    help="leave the serving block out of the default line")
    ap.add_argument("--serving-block-rate", type=float, default=1000.0)
    ap.add_argument("--serving-block-seconds", type=float, default=3.0)
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[100, 300, 1000, 3000, 5000])
    ap.add_argument("--serving-seconds", type=float, default=2.0)
    ap.add_argument("--serving-warmup", type=float, default=0.0,
                    help="seconds of an unreported load at the first rate before the measured ones")
    ap.add_argument("--serving-streams", type=int, default=4)
    ap.add_argument("--serving-layout", default="tensor", choices=["plain", "tensor"],
                    help="resident layout of the served DBs (tensor: the bf16 tensor-core GEMM, twice the bytes)")
    ap.add_argument("--serving-max-batch", type=int, default=32)
    ap.add_argument("--serving-graphs", action="store_true",
                    help="run batches as captured graphs per (database, batch bucket, stream), autotuned")
    ap.add_argument("--serving-graph-gib", type=int, default=16, help="buffers bound to captured graphs, at most")
    ap.add_argument("--serving-big-slots", type=int, default=2,
                    help="streams the 16 GiB database may hold at once (0: no cap)")
    ap.add_argument("--serving-timeout", type=float, default=30.0,
                    help="seconds after which a batch that has not completed fails its requests")
    ap.add_argument("--serving-headline-rate", type=float, default=0.0,
                    help="offered rate whose p99 is the line's value (default: the highest one kept up with)")
    # the budget counts the library's own scratch per query (about 1.06 GiB for the
    # 16 GiB DB in the tensor layout): 32 GiB lets two of its batches of about 15 run
    # at once; 52 GiB (more batches in flight beside the 208 GiB of resident DBs)
    # stalled at 1000 q/s
    ap.add_argument("--serving-scratch-gib", type=int, default=32)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.ntt_sweep:
        return ntt_sweep(args)
    if args.tensor_large:
        return tensor_large_bench(args)
    if args.lwe:
        return lwe_bench(args)
    if args.serving:
        # Batch buffers of very different sizes (up to 8 GiB for the 16 GiB DB) come and
        # go on four streams; torch's stream-ordered allocator serves them without the
        # device-wide synchronisation a caching-allocator release implies.  Measured with
        # the tensor layout at 3000 q/s: 475 q/s with the caching allocator, 1373 with
        # this one.  Only effective before torch initialises CUDA, as here.
        os.environ.setdefault("PYTORCH_CUDA_ALLOC_CONF", "backend:cudaMallocAsync")
        return serving_bench(args)
    if args.impl == "reference":
        reference_arm(args, args.workload)
    else:
        our_arm(args, args.workload)


if __name__ == "__main__":
    main()
