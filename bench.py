#!/usr/bin/env python
"""Throughput of the LSH fingerprint search on GB300: fingerprints/s, bit-exact.

One step = the whole hot path on one station's fingerprints resident in HBM:
Min-Max signatures -> per-table bucket keys -> radix-sorted hash tables ->
occurrence filter -> pair enumeration + vote counting -> canonical (i, j,
votes) list (fast_detect).  The workload is the paper-scale single station:
3 months at 1 s lag (N = 7,776,000 windows), D = 8192, K = 400, Min-Max
b = 100 x r = 4, v = 4, |i - j| <= 10 excluded, 0.5 % occurrence filter,
synthetic (seeded) fingerprints with 2,000 repeating templates and three
periodic noise sources.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun, one rank per GPU) every rank searches its own station
(an independent problem, no data-path collective): weak scaling; the value is
the fingerprints of all ranks over the slowest rank's time.
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
    import synth
    if rank != 0:
        return 0
    w = synth.workload(args.workload)
    n = args.ref_sample
    sw = _sample_workload(w, n)
    times, thr, M = [], 0, 0
    for k in range(args.warmup + args.steps):
        dt, thr, M = oracle_sample(sw, n)
        if k >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.mean(times)
    value = n / (ms / 1000)
    sample = (f"first {n:,} windows of the {w.name} workload (its own filter threshold), whole path "
              f"(keys on {thr} threads, filter, search single-threaded); {M:,} detections")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(w, 1, {"sample_windows": n}),
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
          "k_pairs", "k_vote")


def _kernel_source_hash(rel: str) -> str:
    import hashlib
    return hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16]


def _traffic(kernel: str, units: float):
    """DRAM bytes per launch from the committed ncu capture of this kernel
    (profiles/dram_traffic.json: bytes per unit, scaled to this launch), or
    None when there is none or the kernel's source changed since."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))[kernel]
    except (OSError, ValueError, KeyError):
        return None
    if _kernel_source_hash(rec["source"]) != rec["source_sha256_16"]:
        return None
    return rec["bytes_per_unit"] * units


def kernel_rooflines(w, per, st, peaks, n_sms):
    """Per kernel: live ms per launch, algorithmic bytes per launch and the
    HBM roofline fraction they reach.  Algorithmic bytes (per unit):
      k_sig_walk      read K u16 indices + write b keys  = 2K + 4b  per fingerprint
      radix sort      read key + write (key, id)         = 12       per table entry (all passes together)
      k_pairs_grp<2>  read (key, id) 8 per table entry + write 4 per small-bucket pair (one pass)
      k_warp_vote     read 4 per pair emission + write 5 per kept sparse pair (not counted: small)
      output          write (i, j, votes)                = 9        per detection"""
    N, b, K = w.N, w.b, w.K
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    out = {}

    def put(name, ms, nbytes, single, traffic=None, **extra):
        ach = nbytes / (ms / 1000) / 1e9 if ms > 0 else 0.0
        out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": traffic, "peak_source": src, "algorithmic_bytes": nbytes, "ms": ms,
                     "single_kernel": single, **extra}

    F = b * ((w.r + 1) // 2) if w.kind else b * w.r
    clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    alu_peak = n_sms * 128 * clock  # int32 lanes x clock
    put("k_sig_walk", per["sig"], N * (2 * K + 4 * b), True, _traffic("k_sig_walk", N),
        alu_view={"definition": "direct evaluation: N*K*F hash evaluations x 4 int ops",
                  "ops": N * K * F * 4, "peak_ops_per_s": alu_peak,
                  "time_at_peak_ms": 1000 * N * K * F * 4 / alu_peak})
    passes = max(1, st["sort_passes"])
    put("radix sort", per["sort"], N * b * 12, False, None, passes=passes)
    put("k_pairs_grp<2>", per["k_pairs"], N * b * 8 + st["n_pairs_small"] * 4, True,
        _traffic("k_pairs_grp<2>", N))
    put("k_warp_vote", per["k_vote"], st["n_emissions"] * 4, True, _traffic("k_warp_vote", N))
    put("output", per["output"], st["n_detections"] * 9, False)
    return out


TRAFFIC_KERNELS = {  # kernel-name prefix in the ncu list -> (roofline name, source file)
    "k_sig_walk": ("k_sig_walk", "paper_1803_09835_gb300/csrc/k_sig.cu"),
    "k_pairs_grp<2": ("k_pairs_grp<2>", "paper_1803_09835_gb300/csrc/k_search.cu"),
    "k_warp_vote": ("k_warp_vote", "paper_1803_09835_gb300/csrc/k_search.cu"),
}


def record_traffic(csv_path: str, n_windows: int, command: str, out_path: str | None = None) -> dict:
    """profiles/dram_traffic.json from one ncu --csv capture of
    dram__bytes_read.sum and dram__bytes_write.sum: per kernel of
    TRAFFIC_KERNELS, the first launch's bytes per window of the workload,
    with the hash of the kernel's source file at capture time."""
    import csv
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
        if key is None or (key in seen and seen[key]["id"] != r[ii]):
            continue
        rec = seen.setdefault(key, {"id": r[ii], "read": 0.0, "write": 0.0})
        v = float(r[vi].replace(",", "")) * scale.get(r[ui], 1)
        if r[mi] == "dram__bytes_read.sum":
            rec["read"] = v
        elif r[mi] == "dram__bytes_write.sum":
            rec["write"] = v
    out = {}
    for key, rec in seen.items():
        name, src = TRAFFIC_KERNELS[key]
        out[name] = {"source": src, "source_sha256_16": _kernel_source_hash(src),
                     "bytes_per_unit": (rec["read"] + rec["write"]) / n_windows, "unit": "fingerprint",
                     "captured_on": f"{n_windows:,} windows, first launch", "dram_read_bytes": rec["read"],
                     "dram_write_bytes": rec["write"], "command": command}
    with open(out_path or os.path.join(ROOT, "profiles", "dram_traffic.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    return out


def path_sol(w, per, st, peaks, n_sms, ms_step):
    """Speed-of-light time of the whole path by stage (each stage at the larger
    of its HBM time and, for signatures, the direct-evaluation ALU time), over
    the measured step time."""
    N, b, K = w.N, w.b, w.K
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    clock = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    F = b * ((w.r + 1) // 2) if w.kind else b * w.r
    t = {
        "sig": max(N * (2 * K + 4 * b) / hbm, N * K * F * 4 / (n_sms * 128 * clock)),
        "sort_filter": N * b * 20 / hbm,  # read key 4, write (key, id) 8, read key 4 + id 4 again
        "pairs_votes": st["n_emissions"] * 13 / hbm,
        "output": st["n_detections"] * 9 / hbm,
    }
    tsol = 1000 * sum(t.values())
    return {"t_sol_ms": tsol, "frac": tsol / ms_step, "by_stage_ms": {k: 1000 * v for k, v in t.items()}}


def gpu_arm(args, rank, world, local_rank):
    import numpy as np
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    w = station_workload(args.workload, rank, args.n)
    ld = ((w.K + 7) // 8) * 8
    h_idx = torch.empty((w.N, ld), dtype=torch.uint16, pin_memory=True)
    synth.generate(w, ld=ld, out=h_idx)
    d_idx = h_idx.cuda()
    s = Searcher(w.params())

    def step():
        r = s.detect(d_idx)
        m = r.M
        r.free()
        return m, s.stats()

    acc = {k: 0.0 for k in STAGES}
    counted = {"launches": 0, "on": False}

    def timed_step():
        M, st = step()
        if counted["on"]:
            for k in STAGES:
                acc[k] += st["ms_" + k]
            counted["launches"] += st["n_launches"]
        return M, st

    clocks = Clocks(local_rank)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def start():
        clocks.start()
        counted["on"] = True
        ev0.record()

    def stop():
        ev1.record()
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    ms, (M, last) = timed_steps(timed_step, args.steps, args.warmup, dist, torch.cuda.synchronize, (start, stop))
    clk = clocks.stop()
    launches = counted["launches"]
    ms = max_over_ranks(ms, dist, "cuda")
    n_total = w.N * world
    value = weak_value([w.N] * world, ms)

    # end to end through the host entry point: pinned input in, pinned result out
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    h_i = torch.empty(M, dtype=torch.int32, pin_memory=True)
    h_j = torch.empty(M, dtype=torch.int32, pin_memory=True)
    h_v = torch.empty(M, dtype=torch.uint8, pin_memory=True)
    from paper_1803_09835_gb300 import fast_detect_host
    fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, M)  # warm-up: the library's pool grows once
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        m2 = fast_detect_host(s.ctx, h_idx, w.N, ld, h_i, h_j, h_v, M)
    torch.cuda.synchronize()
    e2e_ms = 1000 * (time.perf_counter() - t0) / e2e_steps
    assert m2 == M
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")

    # roofline of the dominant kernel (live CUDA-event times, algorithmic bytes)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    per = {k: acc[k] / args.steps for k in STAGES}
    kernels = kernel_rooflines(w, per, last, peaks, torch.cuda.get_device_properties(local_rank).multi_processor_count)
    dom = max((k for k in kernels if kernels[k]["single_kernel"]), key=lambda k: kernels[k]["ms"])
    roof = dict(kernels[dom])
    roof["kernel"] = dom
    roof.pop("single_kernel")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(w, world, {"detections_per_station": M}),
            "e2e": {"value": n_total / (e2e_ms / 1000), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": w.N * ld * 2, "d2h_bytes_per_step": M * 9},
            "gpu_launches": launches, "roofline": roof, "clocks": clk,
            "kernels": {k: {kk: v[kk] for kk in ("ms", "bound", "achieved", "frac", "unit")}
                        for k, v in kernels.items()},
            "path_sol": path_sol(w, per, last, peaks, torch.cuda.get_device_properties(local_rank).multi_processor_count,
                                 ms),
            "stage_ms": per,
            "counters": {k: last[k] for k in ("n_dropped", "n_emissions", "n_dense_pairs", "n_groups",
                                              "n_detections", "map_slots", "query_parts", "sort_passes",
                                              "n_long_rows", "n_huge_rows", "max_row", "n_pairs_small",
                                              "n_overflow", "peak_bytes")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, thr, Ms = oracle_sample(w, args.cpu_sample)
        line["cpu_baseline"] = {"value": args.cpu_sample / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": f"first {args.cpu_sample:,} windows of the same workload, whole path "
                                          f"(keys on {thr} threads, filter, search single-threaded), "
                                          f"{dt:.1f} s, {Ms:,} detections"}
    s.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- batched stations

C2_GROUPS = ((12,), (11,), (10,), (9,), (8,), (7,), (6, 1), (5, 2), (4, 3))  # stations by months, ~<= 31M windows


def batch_arm(args):
    """The 12-station workload (stations of 1..12 months, 202,176,000 windows),
    searched as batches of whole stations that fit the device: one
    fast_detect_batch per group, device time by CUDA events, inputs resident.
    The (4, 3)-month group is also run as a batch plan (graph-replayed build,
    autotuned search), and its stations are checked against single-station
    searches (a batch must find exactly what each station finds alone)."""
    import numpy as np
    import torch

    import synth
    from paper_1803_09835_gb300 import Searcher
    base = synth.workload("c2", station=0)
    ld = ((base.K + 7) // 8) * 8
    s = Searcher(dict(base.params(), query_part=args.query_part))
    warm = min(args.warmup, 1)
    groups = C2_GROUPS if not args.n else ((2, 1),)
    if args.groups:
        groups = tuple(tuple(int(m) for m in g.split("+")) for g in args.groups.split(","))
    rows, tot_ms, tot_win, tot_det = [], 0.0, 0, 0
    for grp in groups:
        ws = [synth.workload("c2", station=m - 1) for m in grp]
        if args.n:
            ws = [synth.scaled("c2", args.n * m, station=m - 1) for m in grp]
        t0 = time.perf_counter()
        host = np.concatenate([synth.generate(w, ld=ld) for w in ws])
        gen_s = time.perf_counter() - t0
        d_idx = torch.from_numpy(host).cuda()
        del host
        lens = [w.N for w in ws]
        for _ in range(warm):
            for r in s.detect_batch(d_idx, lens):
                r.free()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        res = s.detect_batch(d_idx, lens)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        det = [r.M for r in res]
        row = {"months": list(grp), "windows": sum(lens), "ms": ms, "detections": det, "gen_s": gen_s}
        if grp == (4, 3) or args.n:
            # exactness across batching: each station alone
            same = True
            off = 0
            for k, w in enumerate(ws):
                alone = s.detect(d_idx[off:off + w.N])
                same &= all(np.array_equal(a, b) for a, b in zip(alone.numpy(), res[k].numpy()))
                alone.free()
                off += w.N
            row["batch_equals_alone"] = bool(same)
            st = torch.cuda.Stream()
            torch.cuda.synchronize()
            plan = s.plan(d_idx, lens, st)
            for r in plan.run():  # first run: the autotuner times its candidates
                r.free()
            torch.cuda.synchronize()
            p0 = time.perf_counter()
            pres = plan.run()
            torch.cuda.synchronize()
            info = plan.info()
            row["plan"] = {"ms_wall": 1000 * (time.perf_counter() - p0), "build_graph_ms": info["build_ms"],
                           "graph_kernels": info["graph_kernels"], "best": info["best"],
                           "same": bool(all(all(np.array_equal(a, b) for a, b in zip(x.numpy(), y.numpy()))
                                            for x, y in zip(pres, res)))}
            for r in pres:
                r.free()
            plan.close()
        for r in res:
            r.free()
        del d_idx
        torch.cuda.empty_cache()
        rows.append(row)
        tot_ms += ms
        tot_win += sum(lens)
        tot_det += sum(det)
        print(json.dumps(row), flush=True)
    line = {"metric": "fingerprints/sec searched, stations batched", "value": tot_win / (tot_ms / 1000),
            "unit": UNIT, "n_gpus": 1, "data": "synthetic", "dtype": "u32",
            "config": {"workload": "c2: 12 stations of 1..12 months (N_s = s x 2,592,000), shared templates",
                       "windows": tot_win, "batches": [list(g) for g in groups], "query_part": args.query_part},
            "ms_total": tot_ms, "detections": tot_det}
    print(json.dumps(line), flush=True)
    s.close()
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
    ap.add_argument("--workload", default="c1")
    ap.add_argument("--n", type=int, default=0, help="override N (windows per station) for quick runs")
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
    ap.add_argument("--batch", action="store_true", help="12-station workload (c2) searched in station batches")
    ap.add_argument("--query-part", type=int, default=4, help="query partitions of the pair buffer for --batch")
    ap.add_argument("--groups", default="", help="--batch station groups by months, e.g. '12,6+1'")
    ap.add_argument("--record-traffic", default="", metavar="CSV",
                    help="write profiles/dram_traffic.json from an ncu dram-bytes capture of this workload")
    ap.add_argument("--record-command", default="", help="the ncu command line to note beside --record-traffic")
    args = ap.parse_args()
    if args.record_traffic:
        w = station_workload(args.workload, 0, args.n)
        print(json.dumps(record_traffic(args.record_traffic, w.N, args.record_command), indent=1))
        return 0
    if args.serving:
        return serving_arm(args)
    if args.batch:
        return batch_arm(args)
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
