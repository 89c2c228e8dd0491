#!/usr/bin/env python
"""Throughput of the LSH fingerprint search on GB300: fingerprints/s, bit-exact.

Headline workload (default): the batched multi-station search -- 12 stations
of 1..12 months at 1 s lag (N_s = s x 2,592,000 windows, 202,176,000 in all),
D = 8192, K = 400, Min-Max b = 100 x r = 4, v = 4, |i - j| <= 10 excluded,
0.5 % occurrence filter per station, 8,000 templates shared across stations
at station offsets of 0..30 windows, periodic noise every 60, 300 and 3600 s.
One step = the whole hot path over all 12 stations, their fingerprints
resident in HBM: Min-Max signatures -> bucket keys -> radix-sorted tables
(10 tables at a time) -> occurrence filter -> pair enumeration + votes ->
canonical (i, j, votes) lists, searched as batches of whole stations
(fast_detect_batch; pairs never cross stations).  Beside it: the same
stations one fast_detect per station ("plain"), the end-to-end figure from
pinned host memory (fast_detect_host, results copied back), and the
single-station 3-month workload (c1) as a diagnostic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun, one rank per GPU) every rank searches its own network
of stations (independent problems, no data-path collective): weak scaling;
the value is the fingerprints of all ranks over the slowest rank's time.
``--impl reference`` times the CPU oracle (plain C, the definition written
out) on a bounded sample of the same workload on this machine's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fingerprints/sec searched (bit-exact) + HBM roofline %; stream p50/p99 ms vs plain"
UNIT = "fingerprints/s"


def workload_config(w, n_gpus, extra=None):
    cfg = {
        "workload": f"{w.name}: {w.N:,} windows/station (1 s lag), D={w.D}, K={w.K}, "
                    f"{'Min-Max' if w.kind else 'MinHash'} b={w.b} x r={w.r}, v={w.v}, excl={w.excl}, "
                    f"occurrence filter {100.0 * w.occ_num / w.occ_den:g}% in > b/2 tables, "
                    f"{w.n_templates} templates, periodic sources {list(w.periods)} s",
        "stations": n_gpus,
        "N_per_station": w.N,
        "l2": "inputs larger than L2 (idx %.1f GB/station), no flush" % (w.N * w.K * 2 / 1e9),
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks

class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg

def oracle_sample(w, n_sample: int):
    """The oracle, as it stands, on the first n_sample windows of the workload."""
    import numpy as np

    import oracle
    import synth
    idx = synth.generate(_sample_workload(w, n_sample), ld=w.K)
    p = w.params()
    t0 = time.perf_counter()
    keys, threads = oracle.keys(p, idx, return_threads=True)
    d = oracle.drop(p, keys)
    i, _, _ = oracle.search(p, keys, d)
    dt = time.perf_counter() - t0
    return dt, threads, len(i)


def _sample_workload(w, n):
    """The first n windows of workload w, exactly: every draw of the generator
    is keyed by window index, and repeats placed beyond n are dropped."""
    from dataclasses import replace
    return replace(w, N=n, place_range=w.place_range or w.N)


def reference_arm(args, rank, world):
    """The oracle, as it stands, on a bounded sample of the workload (its
    first --ref-sample windows; for the 12-station workload, of its
    12-month station), each step one whole-path run on the host cores."""
    import synth
    if rank != 0:
        return 0
    if args.workload == "c2":
        w = c2_stations(0)[11]
        what = "the 12-month station of the 12-station workload"
        cfg = {"workload": "c2: 12 stations of 1..12 months (202,176,000 windows); the oracle runs a bounded "
                           "sample of it", "sample_windows": args.ref_sample}
    else:
        w = synth.workload(args.workload)
        what = f"the {w.name} workload"
        cfg = workload_config(w, 1, {"sample_windows": args.ref_sample})
    n = args.ref_sample
    sw = _sample_workload(w, n)
    times, thr, M = [], 0, 0
    for k in range(args.warmup + args.steps):
        dt, thr, M = oracle_sample(sw, n)
        if k >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.mean(times)
    value = n / (ms / 1000)
    sample = (f"first {n:,} windows of {what} (its own filter threshold), whole path "
              f"(keys on {thr} threads, filter, search single-threaded); {M:,} detections")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ multi-rank plumbing
#
# One rank per GPU, one station per rank (an independent problem): the only
# collectives are the barriers around the timed region and the max of the
# per-rank step times.  The functions below are also driven on CPU ranks
# (gloo) by the tests.

def station_workload(name: str, rank: int, n: int = 0):
    """The workload rank `rank` searches: station `rank` of `name` (own seed)."""
    import synth
    return synth.scaled(name, n, station=rank) if n else synth.workload(name, station=rank)


def timed_steps(step, steps: int, warmup: int, dist=None, sync=None, clock=None):
    """W untimed warm-up steps, then exactly K timed steps bracketed by a
    barrier and a device sync on both sides.  `clock` is a pair of callables
    (start, stop -> ms); the default is the host clock.  Returns ms per step
    on this rank and the outputs of the last step."""
    out = None
    for _ in range(warmup):
        out = step()
    for phase in (0, 1):
        if phase == 1:
            ms = clock[1]() if clock else 1000 * (time.perf_counter() - t0)
        if sync:
            sync()
        if dist:
            dist.barrier()
        if sync:
            sync()
        if phase == 0:
            if clock:
                clock[0]()
            else:
                t0 = time.perf_counter()
            for _ in range(steps):
                out = step()
    return ms / steps, out


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """The largest x over all ranks (x itself on a single rank)."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(n_per_rank, ms_max: float) -> float:
    """Whole-job throughput: the windows of every rank over the slowest rank's time."""
    return sum(n_per_rank) / (ms_max / 1000)


# ------------------------------------------------------------------- GB300 leg

STAGES = ("sig", "sort", "filter", "enum", "dense", "sparse", "output", "pair_count", "pair_emit", "vote",
          "k_pairs", "k_vote", "k_medium", "k_vote_block", "k_count_small", "k_count_medium")

def _kernel_source_hash(rel: str) -> str:
    import hashlib
    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]


def _traffic(kernel: str, key: str):
    """DRAM bytes of a kernel in one step (one search of every station of the
    workload), from the committed ncu record of that kernel on this workload
    (profiles/dram_traffic.json, keyed by workload and windows), or None when
    there is none or the kernel's source changed since.  Records are not
    carried across workload sizes: the pair kernels' misses grow faster than
    their work once their buffers outgrow L2."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[key][kernel]
    except (OSError, ValueError, KeyError, TypeError):
        return None
    if _kernel_source_hash(rec["source"]) != rec["source_sha256_16"]:
        return None
    return rec["bytes_per_run"]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


class KernelBytes:
    """Algorithmic bytes of the heavy kernels, summed over the searches of a
    step (each search's counters).  Per unit:
      k_sig_walk          read K u16 indices + write b keys = 2K + 4b per fingerprint
      radix sort          read key + write (key, id)       = 12 per table entry (all passes together)
      k_pairs_grp         read (key, id) 8 per table entry + write 4 per small-bucket pair
      k_medium_grp        write 4 per medium-bucket pair (its bucket reads are not counted)
      k_pairs_grp count   read (key, id) 8 per table entry
      k_warp_vote         read 4 per pair emission
      output              write (i, j, votes) = 9 per detection
    Table reads repeated by query partitions are overhead, not algorithmic."""

    def __init__(self, w):
        self.w = w
        self.b = {k: 0.0 for k in ("k_sig_walk", "radix sort", "k_pairs_grp", "k_medium_grp", "k_pairs_grp count",
                                   "k_warp_vote", "output")}
        self.units = {}

    def add(self, N, st):
        w, b = self.w, self.b
        for k, v in units_of(st, N).items():
            self.units[k] = self.units.get(k, 0) + v
        b["k_sig_walk"] += N * (2 * w.K + 4 * w.b)
        b["radix sort"] += N * w.b * 12
        b["k_pairs_grp"] += N * w.b * 8 + st["n_pairs_small"] * 4
        b["k_medium_grp"] += (st["n_emissions"] - st["n_pairs_small"]) * 4
        b["k_pairs_grp count"] += N * w.b * 8 if st["ms_k_count_small"] > 0 else 0
        b["k_warp_vote"] += st["n_emissions"] * 4
        b["output"] += st["n_detections"] * 9


KERNEL_MS = {"k_sig_walk": "sig", "radix sort": "sort", "k_pairs_grp": "k_pairs", "k_medium_grp": "k_medium",
             "k_pairs_grp count": "k_count_small", "k_warp_vote": "k_vote", "output": "output"}
SINGLE = {"k_sig_walk", "k_pairs_grp", "k_medium_grp", "k_pairs_grp count", "k_warp_vote"}

WALK_TILE, WALK_BATCH = 32, 8  # fingerprints per walk tile, ranking steps read per batch (k_sig_walk)
SMEM_LOOKUPS_PER_CLK = 32      # conflict-free shared-memory reads per SM and clock (one warp-wide load)


def walk_steps(D: int, K: int, tile: int = WALK_TILE, batch: int = WALK_BATCH) -> float:
    """Expected ranking steps of one k_sig_walk walk, for fingerprints of K
    set bits drawn uniformly from D: a walk over one function's ranking of
    [0, D) stops at the batch of `batch` steps in which the last of the
    tile's `tile` fingerprints is hit.  P(a fingerprint is missed by the
    first s elements) = C(D - K, s) / C(D, s); the walk's length is the
    maximum over the tile of the first-hit positions."""
    miss, m = [1.0], 1.0
    for s in range(1, D + 1):
        m *= max(0.0, D - K - (s - 1)) / (D - (s - 1))
        miss.append(m)
    return batch * sum(1.0 - (1.0 - miss[min(D, x)]) ** tile for x in range(0, D + batch, batch))


def walk_bound(w, ms: float, n_fp: float, sms: int = 152, clk_ghz: float = 2.07) -> dict:
    """k_sig_walk against its own work: shared-memory membership lookups
    (one per walk step: every function's min walk and, for Min-Max, its max
    walk, over each tile of 32 fingerprints) per second, against the SMs'
    conflict-free lookup rate at the nominal clock."""
    nf = w.b * w.r if w.kind == 0 else w.b * ((w.r + 1) // 2)
    walks = nf if w.kind == 0 else 2 * nf
    per_fp = walks * walk_steps(w.D, w.K) / WALK_TILE
    rate = n_fp * per_fp / (ms / 1000) if ms > 0 else 0.0
    peak = sms * SMEM_LOOKUPS_PER_CLK * clk_ghz * 1e9
    return {"bound": "smem lookups", "lookups_per_fingerprint": per_fp, "achieved": rate, "peak": peak,
            "unit": "lookups/s", "frac": rate / peak}


def kernel_rooflines(kb, per, steps, peaks, key=""):
    """Per heavy kernel: live ms per step (CUDA events on the launching
    stream, summed over the step's launches), algorithmic bytes per step and
    the HBM roofline fraction they reach; ``traffic`` is DRAM bytes per step
    from the committed ncu record of that kernel on this workload, or None."""
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    out = {}
    for name, stage in KERNEL_MS.items():
        ms = per[stage]
        nbytes = kb.b[name] / steps
        ach = nbytes / (ms / 1000) / 1e9 if ms > 0 else 0.0
        out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": _traffic(name, key), "peak_source": f"{src} ({hbm:g} GB/s)",
                     "algorithmic_bytes": nbytes, "ms": ms, "single_kernel": name in SINGLE}
    if kb.units.get("fingerprint") and kb.w.K * kb.w.K >= kb.w.D:  # the walk kernel against its own work
        out["k_sig_walk"]["walk"] = walk_bound(kb.w, out["k_sig_walk"]["ms"], kb.units["fingerprint"] / steps)
    return out


def dominant(kernels):
    dom = max((k for k in kernels if kernels[k]["single_kernel"] and kernels[k]["ms"] > 0),
              key=lambda k: kernels[k]["ms"])
    roof = dict(kernels[dom])
    roof["kernel"] = dom
    roof.pop("single_kernel")
    return roof


COUNTERS = ("n_dropped", "n_emissions", "n_dense_pairs", "n_groups", "n_detections", "query_parts", "sort_passes",
            "n_long_rows", "n_huge_rows", "max_row", "n_pairs_small", "n_overflow", "peak_bytes", "max_group",
            "large_min", "dense_fallback")


class Meter:
    """Stage times, launches and counters of the searches inside timed steps."""

    def __init__(self, w):
        self.on = False
        self.acc = {k: 0.0 for k in STAGES}
        self.launches = 0
        self.kb = KernelBytes(w)
        self.last = {}

    def add(self, N, st, key=None):
        """One search of N windows; `key` names it in the line's counters
        (default N: batches of equal length need their own keys)."""
        if not self.on:
            return
        for k in STAGES:
            self.acc[k] += st["ms_" + k]
        self.launches += st["n_launches"]
        self.kb.add(N, st)
        self.last[N if key is None else key] = {**{k: st[k] for k in COUNTERS}, "windows": N}


def _sample_line(w, n, label):
    dt, thr, Ms = oracle_sample(w, n)
    return {"value": n / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"first {n:,} windows of {label} (its own filter threshold), whole path (keys on {thr} "
                      f"threads, filter, search single-threaded), {dt:.1f} s, {Ms:,} detections; the oracle's "
                      f"search cost per window grows with the station length, so the full workload runs slower "
                      f"per window than this sample"}


def station_arm(args, rank, world, local_rank, w, steps, warmup, e2e=True):
    """One station per rank, fast_detect on its fingerprints resident in HBM;
    returns the result line (also the diagnostic single-station figures)."""
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher, fast_detect_host

    dist = None
    if world > 1:
        import torch.distributed as dist
    ld = ((w.K + 7) // 8) * 8
    h_idx = torch.empty((w.N, ld), dtype=torch.uint16, pin_memory=True)
    synth.generate(w, ld=ld, out=h_idx)
    d_idx = h_idx.cuda()
    s = Searcher(w.params())
    meter = Meter(w)

    def step():
        r = s.detect(d_idx)
        m = r.M
        r.free()
        meter.add(w.N, s.stats())
        return m

    clocks = Clocks(local_rank)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def start():
        clocks.start()
        meter.on = True
        ev0.record()

    def stop():
        ev1.record()
        torch.cuda.synchronize()
        meter.on = False
        return ev0.elapsed_time(ev1)

    ms, M = timed_steps(step, steps, warmup, dist, torch.cuda.synchronize, (start, stop))
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    n_total = w.N * world
    line = {"metric": METRIC, "value": weak_value([w.N] * world, ms), "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(w, world, {"detections_per_station": M}),
            "gpu_launches": meter.launches, "clocks": clk}
    if e2e and not args.no_e2e:  # end to end through the host entry point: pinned input in, pinned result out
        e2e_steps = max(1, min(steps, args.e2e_steps))
        h_i = torch.empty(M, dtype=torch.int32, pin_memory=True)
        h_j = torch.empty(M, dtype=torch.int32, pin_memory=True)
        h_v = torch.empty(M, dtype=torch.uint8, pin_memory=True)
        fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, M)  # warm-up: the library's pool grows once
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            m2 = fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, M)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(1000 * (time.perf_counter() - t0) / e2e_steps, dist, "cuda")
        assert m2 == M
        line["e2e"] = {"value": n_total / (e2e_ms / 1000), "unit": UNIT, "ms_per_step": e2e_ms,
                       "h2d_bytes_per_step": w.N * ld * 2, "d2h_bytes_per_step": M * 9}
    per = {k: meter.acc[k] / steps for k in STAGES}
    kernels = kernel_rooflines(meter.kb, per, steps, _peaks(), traffic_key(w.name, w.N))
    line["roofline"] = dominant(kernels)
    line["kernels"] = {k: {kk: v[kk] for kk in ("ms", "bound", "achieved", "frac", "unit", "walk") if kk in v}
                       for k, v in kernels.items()}
    line["stage_ms"] = per
    line["counters"] = meter.last.get(w.N, {})
    s.close()
    return line


def c2_stations(rank: int, n_month: int = 0):
    """Rank `rank`'s network of 12 stations, station s (0-based) covering
    s + 1 months (n_month windows per month for quick runs).  Rank 0 is the
    workload itself; other ranks draw their own stations and templates."""
    from dataclasses import replace

    import synth
    ws = []
    for st in range(12):
        w = synth.workload("c2", station=st) if not n_month else synth.scaled("c2", (st + 1) * n_month, station=st)
        if rank:
            w = replace(w, seed=w.seed + 1000 * rank, tpl_seed=w.tpl_seed + 1000 * rank)
        ws.append(w)
    return ws


C2_GROUPS = ((12,), (11,), (10,), (9,), (8,), (7,), (6, 1), (5, 2), (4, 3))  # stations by months, ~<= 31M windows


def c2_arm(args, rank, world, local_rank):
    """The headline: the 12-station workload, every station's fingerprints
    resident in HBM (161.7 GB), one step = all stations searched as batches
    of whole stations (one fast_detect_batch per batch of C2_GROUPS)."""
    import numpy as np
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher, fast_detect_host

    dist = None
    if world > 1:
        import torch.distributed as dist
    ws = c2_stations(rank, args.n)
    ld = 400
    N_all = sum(w.N for w in ws)
    t0 = time.perf_counter()
    bufs = []  # one device buffer per batch: its stations' rows one after another
    for grp in C2_GROUPS:
        sub = [ws[m - 1] for m in grp]
        d = torch.empty((sum(w.N for w in sub), ld), dtype=torch.int16, device="cuda")
        off = 0
        for w in sub:
            d[off:off + w.N].copy_(torch.from_numpy(synth.generate(w, ld=ld).view(np.int16)))
            off += w.N
        bufs.append((grp, d, [w.N for w in sub]))
    gen_s = time.perf_counter() - t0
    p = dict(ws[0].params(), table_group=10)
    s = Searcher(p)
    meter = Meter(ws[0])
    last_M = {}

    def step():
        tot = 0
        for grp, d, lens in bufs:
            res = s.detect_batch(d, lens)
            meter.add(sum(lens), s.stats(), "+".join(str(m) for m in grp))
            for m, r in zip(grp, res):
                last_M[m] = r.M
                tot += r.M
                r.free()
        return tot

    clocks = Clocks(local_rank)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def start():
        clocks.start()
        meter.on = True
        ev0.record()

    def stop():
        ev1.record()
        torch.cuda.synchronize()
        meter.on = False
        return ev0.elapsed_time(ev1)

    ms, M = timed_steps(step, args.steps, args.warmup, dist, torch.cuda.synchronize, (start, stop))
    clk = clocks.stop()
    ms = max_over_ranks(ms, dist, "cuda")
    value = weak_value([N_all] * world, ms)

    # the plain search: the same stations, one fast_detect per station
    plain_M, plain_ms = {}, 0.0
    for grp, d, lens in bufs:
        off = 0
        for m, n in zip(grp, lens):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r = s.detect(d[off:off + n])
            e1.record()
            torch.cuda.synchronize()
            plain_ms += e0.elapsed_time(e1)
            plain_M[m] = r.M
            r.free()
            off += n
    plain_ms = max_over_ranks(plain_ms, dist, "cuda")

    # a batch plan: the (4 + 3)-month batch's build captured as a CUDA graph,
    # search options autotuned on the first run
    plan_info = None
    if not args.no_plan:
        grp, d, lens = next(b for b in bufs if b[0] == (4, 3))
        st_ = torch.cuda.Stream()
        torch.cuda.synchronize()
        plan = s.plan(d, lens, st_)
        for r in plan.run():
            r.free()
        torch.cuda.synchronize()
        pt = time.perf_counter()
        pres = plan.run()
        torch.cuda.synchronize()
        info = plan.info()
        plan_info = {"batch_months": list(grp), "ms_wall": 1000 * (time.perf_counter() - pt),
                     "build_graph_ms": info["build_ms"], "graph_kernels": info["graph_kernels"],
                     "best": info["best"], "same_counts": [r.M for r in pres] == [last_M[m] for m in grp]}
        for r in pres:
            r.free()
        plan.close()
    del bufs, d
    torch.cuda.empty_cache()

    # end to end through the host entry point, station by station: pinned
    # input in, every detection copied back to pinned host memory
    e2e_ms = h2d = d2h = 0
    if not args.no_e2e:
        nmax = max(w.N for w in ws)
        mmax = max(last_M.values())
        h_idx = torch.empty((nmax, ld), dtype=torch.uint16, pin_memory=True)
        h_i = torch.empty(mmax, dtype=torch.int32, pin_memory=True)
        h_j = torch.empty(mmax, dtype=torch.int32, pin_memory=True)
        h_v = torch.empty(mmax, dtype=torch.uint8, pin_memory=True)
        # largest station first, as the other legs: its warm-up call sizes the
        # context's memory pool once, so no timed call grows it
        for k in sorted(range(len(ws)), key=lambda x: -ws[x].N):
            w = ws[k]
            synth.generate(w, ld=ld, out=h_idx[:w.N])  # drawing the input is not timed
            if w.N == nmax:
                fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, mmax)  # warm-up
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            m = fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, mmax)
            torch.cuda.synchronize()
            e2e_ms += 1000 * (time.perf_counter() - t1)
            assert m == last_M[k + 1]
            h2d += w.N * ld * 2
            d2h += m * 9
        e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
        del h_idx, h_i, h_j, h_v
    s.close()
    torch.cuda.empty_cache()

    per = {k: meter.acc[k] / args.steps for k in STAGES}
    kernels = kernel_rooflines(meter.kb, per, args.steps, _peaks(), traffic_key("c2", N_all))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"c2: 12 stations of 1..12 months at 1 s lag (N_s = s x {ws[0].N:,}), "
                                   f"{N_all:,} windows per network, D={ws[0].D}, K={ws[0].K}, Min-Max b={ws[0].b} "
                                   f"x r={ws[0].r}, v={ws[0].v}, excl={ws[0].excl}, occurrence filter 0.5% per "
                                   f"station, templates shared across stations (offsets 0..30), periodic sources "
                                   f"{list(ws[0].periods)} s",
                       "networks": world, "windows_per_step": N_all * world,
                       "batches_months": [list(g) for g in C2_GROUPS], "table_group": 10,
                       "query_part": "automatic (as many as the memory beside the resident inputs needs)",
                       "l2": f"inputs larger than L2 ({N_all * ld * 2 / 1e9:.1f} GB resident), no flush",
                       "input_generation_s": gen_s, "detections_per_step": M},
            "e2e": {"value": (N_all * world / (e2e_ms / 1000)) if e2e_ms else None, "unit": UNIT,
                    "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "how": "fast_detect_host per station (largest first, after one warm-up call on the largest) from "
                           "pinned host memory, every detection copied back "
                           "(the input's drawing between stations not timed)"},
            "gpu_launches": meter.launches, "roofline": dominant(kernels), "clocks": clk,
            "plain": {"value": N_all * world / (plain_ms / 1000), "unit": UNIT, "ms_per_step": plain_ms,
                      "how": "the same stations, one fast_detect per station, inputs resident",
                      "same_counts_as_batched": plain_M == last_M},
            "plan": plan_info,
            "kernels": {k: {kk: v[kk] for kk in ("ms", "bound", "achieved", "frac", "unit", "algorithmic_bytes", "walk")
                            if kk in v}
                        for k, v in kernels.items()},
            "stage_ms": per,
            "counters_by_batch": {str(n): c for n, c in meter.last.items()},
            "detections_by_station_months": {str(m): last_M[m] for m in sorted(last_M)}}
    return line


def gpu_arm(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    if args.workload == "c2":
        line = c2_arm(args, rank, world, local_rank)
        if not args.no_c1:  # the single-station 3-month workload, as a diagnostic
            import synth
            w1 = station_workload("c1", rank, 0)
            c1 = station_arm(args, rank, world, local_rank, w1, steps=5, warmup=3, e2e=False)
            line["c1"] = {k: c1[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "roofline",
                                              "kernels", "stage_ms", "counters")}
        sample_w = _sample_workload(c2_stations(0)[11], args.cpu_sample)
        label = "the 12-month station of the same workload"
    else:
        w = station_workload(args.workload, rank, args.n)
        line = station_arm(args, rank, world, local_rank, w, args.steps, args.warmup)
        sample_w = _sample_workload(w, args.cpu_sample)
        label = "the same workload"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _sample_line(sample_w, args.cpu_sample, label)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


TRAFFIC_KERNELS = {  # kernel-name prefix in the ncu list -> (roofline name, source file, unit)
    "k_sig_walk": ("k_sig_walk", "paper_1803_09835_gb300/csrc/k_sig.cu", "fingerprint"),
    "k_pairs_grp<2": ("k_pairs_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "small-bucket pair"),
    "k_pairs_grp<1": ("k_pairs_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "small-bucket pair"),
    "k_pairs_grp<0": ("k_pairs_grp count", "paper_1803_09835_gb300/csrc/k_search.cu", "small-bucket pair"),
    "k_medium_grp<2": ("k_medium_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "medium-bucket pair"),
    "k_medium_grp<1": ("k_medium_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "medium-bucket pair"),
    "k_medium_warp<2": ("k_medium_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "medium-bucket pair"),
    "k_medium_warp<1": ("k_medium_grp", "paper_1803_09835_gb300/csrc/k_search.cu", "medium-bucket pair"),
    "k_warp_vote": ("k_warp_vote", "paper_1803_09835_gb300/csrc/k_search.cu", "emission"),
}


def traffic_key(name: str, windows: int) -> str:
    """Key of a workload's DRAM record: its name and windows per step."""
    return f"{name}/{windows}"


def units_of(st: dict, N: int) -> dict:
    """Units of the traffic record in one search, from its counters."""
    return {"fingerprint": N, "small-bucket pair": st["n_pairs_small"],
            "medium-bucket pair": st["n_emissions"] - st["n_pairs_small"], "emission": st["n_emissions"]}


def record_traffic(csv_path: str, line_path: str, command: str, out_path: str | None = None, runs: int = 1) -> dict:
    """profiles/dram_traffic.json from one ncu --csv capture of
    dram__bytes_read.sum and dram__bytes_write.sum over a single-station run
    of bench.py, and that run's own JSON line (its counters): per kernel of
    TRAFFIC_KERNELS, the DRAM bytes of its launches per unit of its work
    (fingerprints, pairs written, emissions voted), with the hash of the
    kernel's source file at capture time.  `runs` = the searches the capture
    covers (warm-up and timed steps; the line's counters are one search's).
    A launch of the pair kernels is scaled by pairs, not windows: their
    bytes follow the pairs they write."""
    import csv
    line = json.loads([x for x in open(line_path) if x.startswith("{")][-1])
    if "counters_by_batch" in line:  # the 12-station step: its batches' units
        N = line["config"]["windows_per_step"]
        wkey = traffic_key("c2", N)
        units = {}
        batches = line["counters_by_batch"]
        for n, cnt in batches.items():
            for k, v in units_of(cnt, cnt.get("windows", int(n) if n.isdigit() else 0)).items():
                units[k] = units.get(k, 0) + v * runs
        if sum(c.get("windows", int(n) if n.isdigit() else 0) for n, c in batches.items()) != N:
            units = {}  # counters of some batches missing: bytes per search only
    else:
        N = line["config"]["N_per_station"]
        wkey = traffic_key(line["config"]["workload"].split(":")[0], N)
        units = {k: v * runs for k, v in units_of(line["counters"], N).items()}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    rows = list(csv.reader(open(csv_path)))
    hdr = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    h = rows[hdr]
    ki, mi, ui, vi, ii = (h.index(x) for x in ("Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "ID"))
    seen = {}
    for r in rows[hdr + 1:]:
        if len(r) <= vi:
            continue
        name = r[ki].replace("void ", "").replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
        name = re.sub(r"\((?:int|bool|unsigned int|long|unsigned long)\)", "", name.replace("unnamed>::", ""))
        name = name.split("(")[0].split("::")[-1]
        key = next((k for k in TRAFFIC_KERNELS if name.startswith(k)), None)
        if key is None:
            continue
        rec = seen.setdefault(TRAFFIC_KERNELS[key][0], {"ids": set(), "read": 0.0, "write": 0.0, "key": key})
        rec["ids"].add(r[ii])
        v = float(r[vi].replace(",", "")) * scale.get(r[ui], 1)
        if r[mi] == "dram__bytes_read.sum":
            rec["read"] += v
        elif r[mi] == "dram__bytes_write.sum":
            rec["write"] += v
    out = {}
    for name, rec in seen.items():
        _, src, unit = TRAFFIC_KERNELS[rec["key"]]
        tot = rec["read"] + rec["write"]
        n = units.get(unit, 0)
        out[name] = {"source": src, "source_sha256_16": _kernel_source_hash(src),
                     "bytes_per_run": tot / runs, "bytes_per_unit": tot / n if n else None,
                     "unit": unit if n else None,
                     "captured_on": f"{N:,} windows, {runs} search(es), {len(rec['ids'])} launch(es)"
                                    + (f", {n:,} {unit}s" if n else ""),
                     "dram_read_bytes": rec["read"], "dram_write_bytes": rec["write"], "command": command}
    path = out_path or os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        every = json.load(open(path))
        every = {k: v for k, v in every.items() if "/" in k}  # records of other workloads stay
    except (OSError, ValueError):
        every = {}
    every[wkey] = out
    with open(path, "w") as f:
        json.dump(every, f, indent=1)
        f.write("\n")
    return out


# ------------------------------------------------------------- parameter sweep

def sweep_arm(args):
    """Bucket statistics and search cost against the number of values per
    table r, on uniform and on imbalanced, correlated fingerprints (§6.3:
    skewed bits make large buckets; more hash values per table shrink them).
    One C1-shaped station of --n windows (default 1,000,000) per setting;
    per table: the bucket pairs sum(s (s - 1) / 2) (the candidates the search
    has to count), their share of all pairs (selectivity), the largest
    bucket and the share of fingerprints in the largest 0.1 % of buckets."""
    from dataclasses import replace

    import numpy as np
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher
    torch.cuda.set_device(0)
    n = args.n or 1_000_000
    base = synth.scaled("c1", n)
    rows = []
    for skew, corr in ((0.0, 0.0), (0.3, 0.0), (0.6, 0.3)):
        w = replace(base, skew=skew, corr=corr)
        d = torch.from_numpy(synth.generate(w, ld=400)).cuda()
        for r in (4, 6, 8):
            p = dict(w.params(), r=r)
            s = Searcher(p)
            sig = s.sig(d)
            tb = s.build_tables(sig)
            keys = tb.skey.view(p["b"], -1)
            pairs, big, top = 0, 0, []
            for t in range(p["b"]):  # bucket sizes of table t from its sorted keys (on the host)
                k = keys[t].cpu().numpy()
                cut = np.flatnonzero(np.diff(k)) + 1
                sizes = np.diff(np.concatenate(([0], cut, [len(k)])))
                pairs += int((sizes.astype(np.int64) * (sizes - 1) // 2).sum())
                big = max(big, int(sizes.max()))
                q = max(1, len(sizes) // 1000)
                top.append(np.sort(sizes)[::-1][:q].sum() / len(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = s.search(tb)
            torch.cuda.synchronize()
            ms = 1000 * (time.perf_counter() - t0)
            st = s.stats()
            row = {"skew": skew, "corr": corr, "r": r, "windows": n, "bucket_pairs": pairs,
                   "selectivity": pairs / (p["b"] * n * (n - 1) / 2), "largest_bucket": big,
                   "top0.1%_bucket_share": float(np.mean(top)), "detections": res.M, "dropped": st["n_dropped"],
                   "search_ms": ms, **{k: st[k] for k in ("n_emissions", "n_dense_pairs", "n_groups", "max_group",
                                                          "n_long_rows", "n_huge_rows", "max_row", "large_min",
                                                          "ms_enum", "ms_dense", "ms_sparse")}}
            print(json.dumps(row), flush=True)
            rows.append(row)
            res.free()
            tb.free()
            s.close()
            del sig
        del d
        torch.cuda.empty_cache()
    return 0


# ------------------------------------------------------------ query-only hashing

def query_arm(args):
    """Query-only hashing (§6.4: hash only the queries, check every other
    item against their buckets) against hashing everything, for a small
    number of queries on a large data set: --queries new windows after an
    N-window C1-shaped history (default 1,000 on 1,000,000, the paper's
    example), occurrence filter off so that both ways define the same list.
    Hashing everything: fast_detect over history + queries, the pairs with j
    among the queries kept.  Query-only: fast_query_only.  Device time by
    CUDA events, mean of --steps runs after --warmup."""
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher
    torch.cuda.set_device(0)
    n0 = args.n or 1_000_000
    nq = args.queries
    w = synth.scaled("c1", n0 + nq, occ_num=0)
    d = torch.from_numpy(synth.generate(w, ld=400)).cuda()
    s = Searcher(w.params())
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        tot, out = 0.0, None
        for k in range(args.warmup + args.steps):
            ev[0].record()
            out = fn()
            ev[1].record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                tot += ev[0].elapsed_time(ev[1])
            if k + 1 < args.warmup + args.steps:
                out.free()
        return tot / args.steps, out

    ms_full, full = timed(lambda: s.detect(d))
    ms_q, q = timed(lambda: s.query_only(d[:n0], d[n0:]))
    fi, fj, fv = full.numpy()
    keep = fj >= n0
    same = all((a[keep] == b).all() if len(b) == keep.sum() else False for a, b in zip((fi, fj, fv), q.numpy()))
    line = {"metric": "query-only hashing vs hashing everything", "unit": "ms", "higher_is_better": False,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": "u32",
            "config": {"workload": f"{n0:,} history windows (C1 shape, filter off) + {nq:,} query windows, "
                                   f"D={w.D}, K={w.K}, Min-Max b={w.b} x r={w.r}, v={w.v}"},
            "hash_everything_ms": ms_full, "query_only_ms": ms_q, "speedup": ms_full / ms_q,
            "query_pairs": q.M, "same_pairs": bool(same)}
    full.free()
    q.free()
    s.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ alignment

def align_arm(args):
    """The steps after the search (§7.1, §7.2) on one 3-month station
    searched three times with independent hash families (its three
    channels): channel level (fast_channel_merge: the lists summed per pair,
    threshold 3v) and station level (fast_station_clusters on the merged
    list).  Device time by CUDA events over --steps runs after --warmup."""
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher
    torch.cuda.set_device(0)
    w = synth.scaled("c1", args.n) if args.n else synth.workload("c1")
    d = torch.from_numpy(synth.generate(w, ld=400)).cuda()
    ctxs, lists = [], []
    for k in range(3):
        s = Searcher(dict(w.params(), seed=w.params()["seed"] + 1000 * k))
        ctxs.append(s)
        lists.append(s.detect(d))
    del d
    torch.cuda.empty_cache()
    s = ctxs[0]
    thr = 3 * w.v
    T = sum(r.M for r in lists)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    t_merge = t_clu = 0.0
    for k in range(args.warmup + args.steps):
        ev[0].record()
        m = s.channel_merge(lists, N=w.N, thr=thr)
        ev[1].record()
        c = s.station_clusters(m, gap=args.gap, width=args.width, min_n=args.min_n)
        ev[2].record()
        torch.cuda.synchronize()
        if k >= args.warmup:
            t_merge += ev[0].elapsed_time(ev[1])
            t_clu += ev[1].elapsed_time(ev[2])
        M, nc = m.M, c.n
        c.free()
        m.free()
    t_merge /= args.steps
    t_clu /= args.steps
    hbm = float(_peaks().get("hbm_gbs", 6800.0))
    merge_bytes = T * 9 + M * 10      # read every channel's (i, j, votes), write (i, j, sim)
    clu_bytes = M * 10 + nc * 48      # read the merged list, write 6 x 8 bytes per cluster
    line = {"metric": "alignment entries/s (channel merge + station clusters)", "unit": "entries/s",
            "value": T / ((t_merge + t_clu) / 1000), "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "data": "synthetic", "dtype": "u32",
            "config": {"workload": f"{w.name}: {w.N:,} windows, three channels = three hash seeds, "
                                   f"merge threshold {thr}, clusters gap={args.gap} width={args.width} "
                                   f"min_n={args.min_n}",
                       "channel_entries": T, "merged_entries": M, "clusters": nc},
            "channel_merge": {"ms": t_merge, "entries_per_s": T / (t_merge / 1000),
                              "roofline": {"bound": "hbm", "achieved": merge_bytes / (t_merge / 1000) / 1e9,
                                           "peak": hbm, "unit": "GB/s",
                                           "frac": merge_bytes / (t_merge / 1000) / 1e9 / hbm,
                                           "algorithmic_bytes": merge_bytes}},
            "station_clusters": {"ms": t_clu, "entries_per_s": M / (t_clu / 1000),
                                 "roofline": {"bound": "hbm", "achieved": clu_bytes / (t_clu / 1000) / 1e9,
                                              "peak": hbm, "unit": "GB/s",
                                              "frac": clu_bytes / (t_clu / 1000) / 1e9 / hbm,
                                              "algorithmic_bytes": clu_bytes}}}
    for r in lists:
        r.free()
    for c_ in ctxs:
        c_.close()
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving leg

def serving_arm(args):
    """Streaming workload: resident station histories, Poisson arrivals of
    batches (open loop), p50/p99 latency submit -> result, windows/s; the
    plain search (tables rebuilt for history + batch) per request beside it."""
    import numpy as np
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher, Server

    torch.cuda.set_device(0)
    n_st = args.stations
    n_req = int(args.rate * args.duration)
    t_arr, st_of, size = synth.requests(n_req, args.rate, n_stations=n_st)
    per_st = [int(size[st_of == s].sum()) for s in range(n_st)]
    base = synth.workload("c3") if not args.n else synth.scaled("c3", args.n)
    N0 = base.N
    ld = ((base.K + 7) // 8) * 8
    srv = Server(base.params(), n_st, max_stream_windows=max(per_st) + 1, hbm_budget_bytes=args.budget_gb << 30)
    idx = []
    t0 = time.perf_counter()
    from dataclasses import replace
    for s in range(n_st):
        # the station's 3-month history followed by the windows its requests carry
        ws = synth.scaled("c3", args.n, station=s) if args.n else synth.workload("c3", station=s)
        w = replace(ws, N=N0 + per_st[s])
        a = synth.generate(w, ld=ld)
        srv.load_history(s, a[:N0])
        idx.append(a)
    load_s = time.perf_counter() - t0
    # open-loop replay
    cursor = [N0] * n_st
    ids = []
    start = time.perf_counter()
    for q in range(n_req):
        now = time.perf_counter() - start
        if t_arr[q] > now:
            time.sleep(t_arr[q] - now)
        s = int(st_of[q])
        sl = idx[s][cursor[s]:cursor[s] + int(size[q])]
        ids.append(srv.submit(s, sl))
        cursor[s] += int(size[q])
    results = [srv.wait(r) for r in ids]
    end = time.perf_counter()
    lat = np.array([srv.latency(r) for r in ids]) * 1000
    windows = int(size.sum())
    # plain search per request: tables rebuilt over history + every earlier batch + the batch
    plain_ms, plain_win, plain_ok = [], [], True
    pl = Searcher(base.params())
    cur0 = N0
    for q in [q for q in range(n_req) if st_of[q] == 0][:args.plain_requests]:
        n = int(size[q])
        hist = torch.from_numpy(idx[0][:cur0 + n]).cuda()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = pl.detect(hist)
        gi, gj, gv = r.numpy()
        torch.cuda.synchronize()
        plain_ms.append(1000 * (time.perf_counter() - t1))
        plain_win.append(n)
        r.free()
        keep = gj >= cur0
        first, si, sj, sv = results[q]
        plain_ok &= first == cur0 and np.array_equal(gi[keep], si) and np.array_equal(gj[keep], sj) \
            and np.array_equal(gv[keep], sv)
        cur0 += n
        del hist
    pl.close()
    srv.close()
    line = {"metric": "stream p50/p99 ms vs plain", "value": windows / (end - start), "unit": "windows/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "u32",
            "config": {"workload": f"c3: {n_st} stations x {N0:,} history windows resident, Poisson {args.rate:g} req/s "
                                   f"open loop for {args.duration:g} s, batches log-U[60,3600] windows",
                       "requests": n_req, "windows": windows, "budget_gb": args.budget_gb,
                       "history_load_s": load_s},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "plain": {"requests": len(plain_ms), "p50_ms": float(np.median(plain_ms)) if plain_ms else None,
                      "windows_per_s": float(sum(plain_win) / (sum(plain_ms) / 1000)) if plain_ms else None,
                      "same_as_stream": bool(plain_ok)},
            "detections": int(sum(len(r[1]) for r in results))}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    ap.add_argument("--workload", default="c2", help="c2 (12 stations, the default), or one station: c0, c1")
    ap.add_argument("--n", type=int, default=0,
                    help="quick runs: windows per station (one station) or per month (c2)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-sample", type=int, default=300_000)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", action="store_true", help="streaming workload (c3) instead of the batch search")
    ap.add_argument("--stations", type=int, default=12)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--duration", type=float, default=5.0)
    ap.add_argument("--budget-gb", type=int, default=150)
    ap.add_argument("--plain-requests", type=int, default=3)
    ap.add_argument("--query", action="store_true", help="query-only hashing vs hashing everything")
    ap.add_argument("--queries", type=int, default=1000)
    ap.add_argument("--align", action="store_true", help="channel merge + station clusters on three searches")
    ap.add_argument("--gap", type=int, default=5)
    ap.add_argument("--width", type=int, default=3)
    ap.add_argument("--min-n", type=int, default=2)
    ap.add_argument("--sweep", action="store_true", help="bucket statistics vs r on uniform and skewed fingerprints")
    ap.add_argument("--no-c1", action="store_true", help="skip the single-station diagnostic beside the headline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host memory) leg of the headline")
    ap.add_argument("--no-plan", action="store_true", help="skip the batch-plan leg of the headline")
    ap.add_argument("--record-traffic", default="", metavar="CSV",
                    help="write profiles/dram_traffic.json from an ncu dram-bytes capture of this workload")
    ap.add_argument("--record-line", default="", help="the JSON line of the captured run (its counters)")
    ap.add_argument("--record-runs", type=int, default=1, help="searches the capture covers")
    ap.add_argument("--record-command", default="", help="the ncu command line to note beside --record-traffic")
    args = ap.parse_args()
    if args.record_traffic:
        print(json.dumps(record_traffic(args.record_traffic, args.record_line, args.record_command,
                                        runs=args.record_runs), indent=1))
        return 0
    if args.serving:
        return serving_arm(args)
    if args.sweep:
        return sweep_arm(args)
    if args.align:
        return align_arm(args)
    if args.query:
        return query_arm(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = gpu_arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
