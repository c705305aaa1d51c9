#!/usr/bin/env python3
"""Benchmark of the GB300 string sample sort.

One step = one complete sort (every distribution round, base case and LCP
pass) of one workload that is already resident in device memory, run as
one launch of the library's CUDA graph (options.graph = 1).  The default
workload is 16M URL-like strings (about 0.97 GB of characters, larger than
the 129 MB L2, so no flush is needed between steps).

Prints one JSON line: sorted strings/s over all ranks, plus
  roofline      the dominant kernel's algorithmic bytes / its average launch
                time against the measured HBM copy bandwidth; the launch
                times come from a second timed region of the same sorts with
                the rounds driven from the host and CUDA events recorded by
                the library around every launch on its stream
                (profiled_pass); traffic = the committed ncu DRAM bytes per
                string for the current kernel source, else null
  cpu_baseline  the CPU oracle timed on this host (single thread)
  e2e           the same metric through sss_sort_host: pinned host buffers,
                copies to and from the device inside the timed region
  clocks        SM clocks and throttle reasons sampled during the timed steps
Under torchrun each rank sorts its own replica (no data exchange).

--impl reference times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import gc
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

WORKLOAD_TEXT = {
    "url-16m": "16M URL-like strings: 2,000 Zipf(1.1) hosts + 1-6 Zipf(1.1) path segments, mean 60 B",
    "dna-20m": "20M DNA strings: 64 chars over ACGT from an order-3 Markov chain, 10% exact duplicates",
    "uniform-100k": "100k strings, lengths uniform 8-20, bytes uniform a-z",
    "url-64m": "64M URL-like strings as url-16m (about 3.9 GB of characters)",
}
SCATTER_BYTES_PER_STRING = 26   # read bucket id 2 + key 8 + index 4, write key 8 + index 4
MEDIUM_BYTES_PER_STRING = 24    # read key 8 + index 4, write key 8 + index 4 (bucket ids in shared memory)
REFILL_BYTES = 16               # offset 8 + key word 8, per key word gathered again
CLASSIFY_BYTES_PER_STRING = 10  # read key 8, write bucket id 2
BASE_BYTES_PER_STRING = 20      # read key 8 + index 4, write perm 4 + lcp 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="url-16m", choices=sorted(gen.WORKLOADS))
    ap.add_argument("--mode", default="plain", choices=["plain", "learned"])
    ap.add_argument("--e2e-steps", type=int, default=9)
    ap.add_argument("--cpu-sample", type=int, default=4_000_000,
                    help="strings of the workload the CPU oracle sorts for its baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle child (no D, no cpu_baseline)")
    ap.add_argument("--n", type=int, default=None,
                    help="sort only the first n strings of the workload's generator (profiling runs)")
    ap.add_argument("--legs", default="host,keys8,equal,learned,batched,alphabet,uniform,literal",
                    help="extra measurements beside the headline: host,keys8,equal,learned,batched,alphabet,"
                         "uniform,literal (or none)")
    return ap.parse_args()


# ------------------------------------------------------------------ oracle child

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_child(workload: str, sample: int, n, q):
    """Runs in a spawned process: D of the whole workload, and the oracle's
    time on a bounded sample of it, single-threaded and on every host core
    (sample-cut ranges sorted on threads of their own)."""
    import oracle
    try:
        s = gen.workload(workload, n=n)
        m = min(sample, s.n)
        sub = gen.workload(workload, n=m) if m < s.n else s
        t0 = time.perf_counter()
        perm, lcp = oracle.sort(sub.chars, sub.offsets)
        t = time.perf_counter() - t0
        cores = host_cores()
        t0 = time.perf_counter()
        oracle.sort_parallel(sub.chars, sub.offsets, cores)
        tp = time.perf_counter() - t0
        if m < s.n:
            perm, lcp = oracle.sort_parallel(s.chars, s.offsets, cores)
        D = oracle.dist_prefix(s.chars, s.offsets, perm, lcp)
        q.put({"D": int(D), "N": int(s.total), "cpu_s": t, "cpu_par_s": tp, "cpu_cores": cores, "cpu_n": m,
               "n": s.n})
    except Exception as e:  # reported, never fatal to the GPU measurement
        q.put({"error": repr(e)})


def start_oracle_child(args):
    if args.no_cpu:
        return None, None
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_child, args=(args.workload, args.cpu_sample, args.n, q), daemon=True)
    p.start()
    return p, q


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: str):
        self.gpu = gpu
        self.proc = None
        self.out = ""

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", self.gpu], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.out, _ = self.proc.communicate()
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def visible_gpu(local_rank: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p]
        if local_rank < len(parts):
            return parts[local_rank]
    return str(local_rank)


# ------------------------------------------------------------------ roofline inputs

def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for f in ("sss_kernels.cu", "sss_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1305_1157_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per string of `kernel` from the committed ncu summary of
    this workload, if it was captured on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        vals = {}
        with open(p) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    vals[k.strip()] = v.strip()
        if vals.get("source_sha256_16") != kernel_source_sha():
            return None
        return float(vals["dram_bytes_per_string"])
    except Exception:
        return None


def host_link(torch, stream, dev, h_chars, h_perm, chars, perm, e2e, sort_ms):
    """The host link's copy rates (the step's own pinned buffers, copy engine
    on the bench stream, best of 3) and the end-to-end time they leave: the
    step's uploads and downloads at those rates plus the device-timed sort.
    The entry point uploads before it sorts (the root sample needs every
    string), so that sum is the floor of its end-to-end time."""
    def best(dst, src):
        ts = []
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            with torch.cuda.stream(stream):
                dst.copy_(src, non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return min(ts)
    up = best(chars, h_chars)
    down = best(h_perm, perm)
    h2d_gbs = h_chars.numel() / up / 1e6
    d2h_gbs = 4 * h_perm.numel() / down / 1e6
    copy_ms = e2e["h2d_bytes_per_step"] / h2d_gbs / 1e6 + e2e["d2h_bytes_per_step"] / d2h_gbs / 1e6
    return {"h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs, "copy_ms": copy_ms, "floor_ms": copy_ms + sort_ms,
            "note": "copies at the measured link rates plus the device-timed sort"}


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank):
    """The CPU oracle as it stands, on every host core of rank 0's machine
    (sample-cut ranges, each sorted by the multikey quicksort on a thread of
    its own, then the LCP scan), on a bounded sample of the workload; each
    step sorts the sample once, and the line reports the median step."""
    if rank != 0:
        return 0
    import oracle
    m = min(args.cpu_sample, gen.WORKLOADS[args.workload]["n"])
    sub = gen.workload(args.workload, n=m)
    cores = host_cores()
    steps = max(1, args.steps)
    for _ in range(max(0, min(args.warmup, 3))):
        oracle.sort_parallel(sub.chars, sub.offsets, cores)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle.sort_parallel(sub.chars, sub.offsets, cores)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    v = m / t
    sample = (f"first {m} strings of the {args.workload} workload per step (same generator and seed), "
              f"{cores} host threads")
    line = {"impl": "reference", "metric": "sorted strings/s", "value": v, "unit": "strings/s", "n_gpus": 0,
            "steps": steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOAD_TEXT.get(args.workload, ""),
                       "n": m},
            "cpu_baseline": {"value": v, "unit": "strings/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "strings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ extra legs

def reduce_max(value: float, dist, device) -> float:
    """The largest of each rank's value (the slowest rank's time); the value
    itself without a process group.  device: where the collective's tensor
    lives (the rank's GPU under NCCL, the CPU under gloo)."""
    if not dist:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _step_times(torch, stream, dev, fn, steps, dist, after=None):
    """ms of each of `steps` calls of fn (a CUDA event pair around each call
    on stream), bracketed by a barrier and a synchronize on both sides.
    after(i), if given, runs on the host after call i (not between its
    events' records on the device, which the host does not wait for)."""
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
        if after:
            after(i)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    return [a.elapsed_time(b) for a, b in ev]


def _timed(torch, stream, dev, fn, steps, dist):
    """Median ms per call of fn over `steps` calls, max over ranks."""
    t = _step_times(torch, stream, dev, fn, max(1, steps), dist)
    return reduce_max(statistics.median(t), dist, dev)


def leg_host(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world, dist):
    """The same sort with the rounds driven from the host (one header
    readback per round, no kernel timing) instead of one graph launch."""
    o = sss.sss_get_options()
    saved = o.graph
    o.graph, o.profile = 0, 0
    sss.sss_set_options(o)
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for _ in range(max(2, args.warmup)):
        fn()
    ms = _timed(torch, stream, dev, fn, args.steps, dist)
    st = sss.sss_get_last_stats()
    o.graph = saved
    sss.sss_set_options(o)
    return {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": args.steps,
            "gpu_launches_per_step": int(st.launches), "rounds": int(st.rounds)}


def leg_keys8(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world, dist):
    """Graph form with one-word keys (w = 8 characters, the paper's key)
    instead of two-word keys."""
    o = sss.sss_get_options()
    saved = o.key_bytes
    o.graph, o.profile, o.key_bytes = 1, 0, 8
    sss.sss_set_options(o)
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for _ in range(max(2, args.warmup)):
        fn()
    steps = max(3, args.steps // 2)
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    o.graph, o.key_bytes = 0, saved
    sss.sss_set_options(o)
    return {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
            "key_bytes": 8, "gpu_launches_per_step": int(st.launches), "rounds": int(st.rounds)}


def leg_equal(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world, dist):
    """Graph form with the pS5-Equal classifier (equality test at every tree
    node, early exit) instead of pS5-Unroll."""
    o = sss.sss_get_options()
    saved = o.classifier
    o.graph, o.profile, o.classifier = 1, 0, 1
    sss.sss_set_options(o)
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for _ in range(max(2, args.warmup)):
        fn()
    steps = max(3, args.steps // 2)
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    o.graph, o.classifier = 0, saved
    sss.sss_set_options(o)
    return {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
            "classifier": "pS5-Equal", "key_bytes": int(o.key_bytes), "gpu_launches_per_step": int(st.launches),
            "rounds": int(st.rounds)}


def leg_learned(sss, torch, stream, dev, args, world, dist):
    """Learned bucket proposal (fitted CDF, exact verify, tree fallback) on the
    64M-string URL workload, beside the plain tree classifier with the same
    one-word keys on the same input (host-driven rounds both)."""
    s = gen.workload("url-64m")
    n = s.n
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    saved = sss.sss_get_options()
    o = sss.sss_options.from_buffer_copy(saved)
    o.graph, o.profile, o.key_bytes = 0, 0, 8
    sss.sss_set_options(o)
    steps = max(3, args.steps // 6)
    out = {"workload": WORKLOAD_TEXT["url-64m"], "n": n, "chars_bytes": int(s.total)}
    # the plain sort in its headline form (graph, default key width) on the same input
    g = sss.sss_options.from_buffer_copy(saved)
    g.graph, g.profile = 1, 0
    sss.sss_set_options(g)
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for _ in range(max(2, args.warmup)):
        fn()
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    out["graph_form"] = {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
                         "key_bytes": int(g.key_bytes), "rounds": int(st.rounds),
                         "gpu_launches_per_step": int(st.launches)}
    sss.sss_set_options(o)
    for name, fn in (("tree", lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)),
                     ("learned", lambda: sss.sss_sort_learned(chars, offsets, n, perm, lcp, stream))):
        for _ in range(max(2, args.warmup)):
            fn()
        ms = _timed(torch, stream, dev, fn, steps, dist)
        st = sss.sss_get_last_stats()
        # per-kernel split of one profiled run
        o.profile = 1
        sss.sss_set_options(o)
        fn()
        torch.cuda.synchronize(dev)
        prof = sss.sss_get_last_stats().as_dict()["profile"] or {}
        o.profile = 0
        sss.sss_set_options(o)
        r = {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
             "classify_ms": prof.get("classify", {}).get("ms"), "scatter_ms": prof.get("scatter", {}).get("ms")}
        if name == "learned":
            rk, rm = list(st.round_learned_keys), list(st.round_learned_misses)
            r.update({"proposals": int(st.learned_keys), "misses": int(st.learned_misses),
                      "models": int(st.learned_models),
                      "round_miss_rate": [round(rm[i] / rk[i], 4) for i in range(min(int(st.rounds), 64)) if rk[i]],
                      "round_proposals": [int(rk[i]) for i in range(min(int(st.rounds), 64)) if rk[i]],
                      "miss_rate": (st.learned_misses / st.learned_keys) if st.learned_keys else None,
                      "fit_ms": prof.get("learned", {}).get("ms"),
                      "cdf_segments": int(o.cdf_segments), "cdf_steps": int(o.cdf_steps)})
        out[name] = r
    sss.sss_set_options(saved)
    del chars, offsets, perm, lcp
    torch.cuda.empty_cache()
    return out


def leg_alphabet(sss, torch, stream, dev, args, world, dist):
    """Alphabet compression (App. A.2) on the 20M-string DNA workload: graph
    form with the strings rewritten 3 characters per byte (sigma' = 4) beside
    the same sort on the plain strings."""
    s = gen.workload("dna-20m")
    n = s.n
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    saved = sss.sss_get_options()
    o = sss.sss_options.from_buffer_copy(saved)
    steps = max(3, args.steps // 4)
    out = {"workload": WORKLOAD_TEXT["dna-20m"], "n": n, "chars_bytes": int(s.total)}
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for name, alpha in (("plain", 0), ("compressed", 1)):
        o.graph, o.profile, o.alphabet = 1, 0, alpha
        sss.sss_set_options(o)
        for _ in range(max(2, args.warmup)):
            fn()
        ms = _timed(torch, stream, dev, fn, steps, dist)
        st = sss.sss_get_last_stats()
        # per-kernel split of one profiled (host-driven) run
        o.graph, o.profile = 0, 1
        sss.sss_set_options(o)
        fn()
        torch.cuda.synchronize(dev)
        prof = sss.sss_get_last_stats().as_dict()["profile"] or {}
        out[name] = {"value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
                     "rounds": int(st.rounds), "gpu_launches_per_step": int(st.launches),
                     "alphabet_symbols": int(st.alphabet_symbols), "chars_per_byte": max(1, int(st.alphabet_group)),
                     "profiled_ms": {k: round(v["ms"], 4) for k, v in prof.items() if v["launches"]}}
    sss.sss_set_options(saved)
    del chars, offsets, perm, lcp
    torch.cuda.empty_cache()
    return out


def leg_batched(sss, torch, stream, dev, args, world, dist):
    """10,000 independent sets: one graph launch (autotuned on a tuning batch
    of the same shape, other seed) versus one sss_sort launch per set."""
    import tempfile
    w = gen.BATCH_WORKLOADS["sets-10k"]
    tune = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"] + 1000)
    real = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"])

    def put(b):
        s = b.strings
        return (torch.from_numpy(s.chars).to(dev), torch.from_numpy(s.offsets.view(np.int64)).to(dev),
                torch.empty(s.n, dtype=torch.int32, device=dev), torch.empty(s.n, dtype=torch.int32, device=dev))

    saved = sss.sss_get_options()
    t_chars, t_off, t_perm, t_lcp = put(tune)
    with tempfile.TemporaryDirectory() as d:
        best, tune_ms = sss.sss_autotune_batched(t_chars, t_off, tune.strings.n, tune.set_begin, w["num_sets"],
                                                 t_perm, t_lcp, os.path.join(d, "autotune.jsonl"), stream)
    del t_chars, t_off, t_perm, t_lcp
    chars, off, perm, lcp = put(real)
    n = real.strings.n
    fn = lambda: sss.sss_sort_batched(chars, off, n, real.set_begin, w["num_sets"], perm, lcp, stream)
    for _ in range(2):
        fn()
    steps = max(3, args.steps // 4)
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    # one launch sequence per set (host-driven rounds), all sets once
    sss.sss_set_options(saved)
    sb = real.set_begin.astype(np.int64)

    def per_set():
        for j in range(w["num_sets"]):
            lo, hi = int(sb[j]), int(sb[j + 1])
            sss.sss_sort(chars, off[lo:], hi - lo, perm[lo:], lcp[lo:], stream)

    per_set()
    ms_ps = _timed(torch, stream, dev, per_set, 1, dist)
    return {"workload": "sets-10k: 10,000 sets, sizes log-uniform 100-4000, kinds uniform over "
                        "uniform/url/dna, seed 5", "n": n, "chars_bytes": int(real.strings.total),
            "value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
            "graph_launches_per_step": 1, "kernel_launches_per_step": int(st.launches),
            "per_set_value": n * world / (ms_ps * 1e-3), "per_set_ms": ms_ps,
            "speedup_vs_per_set": ms_ps / ms,
            "tuned": {"k_max": int(best.k_max), "base_threshold": int(best.base_threshold),
                      "medium_threshold": int(best.medium_threshold), "chunk": int(best.chunk),
                      "key_bytes": int(best.key_bytes), "classifier": int(best.classifier),
                      "tuning_ms": tune_ms}}


def leg_uniform(sss, torch, stream, dev, args, world, dist):
    """The small workload (100k strings of 8-20 letters, 1.5 MB:
    it lives in L2 and the sort is bound by launch and round latency, so it
    is reported beside the headline, not as one), graph form."""
    s = gen.workload("uniform-100k")
    n = s.n
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    saved = sss.sss_get_options()
    o = sss.sss_options.from_buffer_copy(saved)
    o.graph, o.profile = 1, 0
    sss.sss_set_options(o)
    fn = lambda: sss.sss_sort(chars, offsets, n, perm, lcp, stream)
    for _ in range(max(3, args.warmup)):
        fn()
    steps = max(5, args.steps)
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    sss.sss_set_options(saved)
    return {"workload": WORKLOAD_TEXT["uniform-100k"], "n": n, "chars_bytes": int(s.total),
            "value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
            "rounds": int(st.rounds), "gpu_launches_per_step": int(st.launches),
            "l2": "inputs fit in L2 (no flush): a side figure, not a headline"}


def leg_literal(sss, torch, stream, dev, args, world, dist):
    """The sets-literal batch: 10,000 sets, sizes log-uniform in [100, 1M]
    (1.09 G strings, about 51 GB of characters), one graph launch with the
    default options, against one sss_sort call per set (host-driven rounds),
    all sets once."""
    w = gen.BATCH_WORKLOADS["sets-literal"]
    sizes, _ = gen.batch_sizes(w["num_sets"], w["lo"], w["hi"], w["seed"])
    n = int(sizes.sum())
    torch.cuda.empty_cache()
    sss.sss_release()
    free, _ = torch.cuda.mem_get_info(dev)
    need = 52e9 + 16 * n + sss.sss_workspace_size(n)
    if free < need:
        return {"skipped": f"needs about {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free"}
    t0 = time.perf_counter()
    b = gen.generate_batch(w["num_sets"], w["lo"], w["hi"], w["seed"])
    gen_s = time.perf_counter() - t0
    s = b.strings
    chars = torch.from_numpy(s.chars).to(dev)
    off = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    saved = sss.sss_get_options()
    o = sss.sss_options.from_buffer_copy(saved)
    o.profile = 0
    sss.sss_set_options(o)
    fn = lambda: sss.sss_sort_batched(chars, off, n, b.set_begin, w["num_sets"], perm, lcp, stream)
    fn()
    steps = max(3, min(5, args.steps))
    ms = _timed(torch, stream, dev, fn, steps, dist)
    st = sss.sss_get_last_stats()
    sb = b.set_begin.astype(np.int64)

    def per_set():
        for j in range(w["num_sets"]):
            lo, hi = int(sb[j]), int(sb[j + 1])
            sss.sss_sort(chars, off[lo:], hi - lo, perm[lo:], lcp[lo:], stream)

    o.graph = 0
    sss.sss_set_options(o)
    ms_ps = _timed(torch, stream, dev, per_set, 1, dist)
    sss.sss_set_options(saved)
    out = {"workload": "sets-literal: 10,000 sets, sizes log-uniform 100-1,000,000, kinds uniform over "
                       "uniform/url/dna, seed 5", "n": n, "chars_bytes": int(s.total),
           "largest_set": int(sizes.max()), "generate_s": gen_s,
           "value": n * world / (ms * 1e-3), "unit": "strings/s", "ms_per_step": ms, "steps": steps,
           "graph_launches_per_step": 1, "kernel_launches_per_step": int(st.launches), "rounds": int(st.rounds),
           "options": "defaults (no autotuning: a tuning batch of this size would be another 51 GB)",
           "per_set_value": n * world / (ms_ps * 1e-3), "per_set_ms": ms_ps, "speedup_vs_per_set": ms_ps / ms}
    del chars, off, perm, lcp, b
    torch.cuda.empty_cache()
    sss.sss_release()
    return out


# ------------------------------------------------------------------ gpu arm

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    child, q = (None, None)
    if rank == 0:
        child, q = start_oracle_child(args)  # spawned before any CUDA call

    import torch
    import paper_1305_1157_gb300 as sss
    from paper_1305_1157_gb300 import build as sbuild

    sbuild.build()
    sss.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    s = gen.workload(args.workload, n=args.n)
    n = s.n
    chars = torch.from_numpy(s.chars).to(dev)
    offsets = torch.from_numpy(s.offsets.view(np.int64)).to(dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sort_fn = sss.sss_sort_learned if args.mode == "learned" else sss.sss_sort

    # the headline form: each sort is one launch of the library's cached CUDA
    # graph (device-side round loop, no host round-trip per round)
    opts = sss.sss_get_options()
    opts.profile, opts.graph = 0, 1
    sss.sss_set_options(opts)
    for _ in range(args.warmup):
        sort_fn(chars, offsets, n, perm, lcp, stream)
    torch.cuda.synchronize(dev)

    launches = [0]
    clocks = ClockSampler(visible_gpu(local_rank))
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.2)

    def count_launches(_i):
        launches[0] += sss.sss_get_last_stats().launches

    step_ms = _step_times(torch, stream, dev, lambda: sort_fn(chars, offsets, n, perm, lcp, stream), args.steps,
                          dist, after=count_launches)
    # the median step (max over ranks) is the headline; the mean beside it
    ms = reduce_max(statistics.median(step_ms), dist, dev)
    ms_mean = reduce_max(sum(step_ms) / len(step_ms), dist, dev)

    # second timed region, per-kernel times: the same sorts with the rounds
    # driven from the host and CUDA events around every kernel launch on the
    # stream it runs on (the roofline and the kernel split come from here)
    opts.graph, opts.profile = 0, 1
    sss.sss_set_options(opts)
    prof_ms = np.zeros(len(sss.K_CLASSES))
    prof_launches = np.zeros(len(sss.K_CLASSES), dtype=np.int64)
    large_strings = large_refills = medium_strings = medium_refills = base_strings = 0
    # a single sort above the medium threshold classifies its root round while
    # k_init_classify builds the records (class "init"), not in k_classify
    root_fused = args.mode != "learned" and n > int(opts.medium_threshold)
    fused_root_strings = 0
    sort_fn(chars, offsets, n, perm, lcp, stream)  # warm the host-driven form
    torch.cuda.synchronize(dev)
    p_start = torch.cuda.Event(enable_timing=True)
    p_end = torch.cuda.Event(enable_timing=True)
    p_start.record(stream)
    for _ in range(args.steps):
        sort_fn(chars, offsets, n, perm, lcp, stream)
        st = sss.sss_get_last_stats()
        prof_ms += np.array(list(st.prof_ms))
        prof_launches += np.array(list(st.prof_launches))
        large_strings += st.round_strings - st.medium_strings
        if root_fused and st.rounds:
            fused_root_strings += st.round_active[0]
        large_refills += st.refilled_strings - st.medium_refilled_strings
        medium_strings += st.medium_strings
        medium_refills += st.medium_refilled_strings
        base_strings += st.base_strings
        last_stats = st.as_dict()
    p_end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms_profiled = p_start.elapsed_time(p_end) / args.steps
    opts.profile = 0
    sss.sss_set_options(opts)

    # the host-side oracle run ends before the end-to-end timing: its threads
    # would compete with the uploads for the host's memory bandwidth
    oracle_info = None
    if child is not None:
        try:
            oracle_info = q.get(timeout=900)
        except Exception as e:
            oracle_info = {"error": repr(e)}
        child.join(timeout=10)

    # end to end through the host-buffer entry point
    e2e = None
    if args.e2e_steps > 0:
        h_chars = torch.from_numpy(s.chars).pin_memory()
        h_off = torch.from_numpy(s.offsets.view(np.int64)).pin_memory()
        h_perm = torch.empty(n, dtype=torch.int32).pin_memory()
        h_lcp = torch.empty(n, dtype=torch.int32).pin_memory()
        sss.sss_sort_host(h_chars, len(s.chars), h_off, n, h_perm, h_lcp)  # warm the io buffers
        if dist:
            dist.barrier()
        # each call timed on the host clock (it returns after its downloads);
        # the median call, as for the headline, with the mean and the
        # slowest beside it
        calls = []
        gc_was_on = gc.isenabled()
        gc.disable()  # no collector pause inside a host-timed call
        try:
            for _ in range(args.e2e_steps):
                t0 = time.perf_counter()
                sss.sss_sort_host(h_chars, len(s.chars), h_off, n, h_perm, h_lcp)
                calls.append(time.perf_counter() - t0)
        finally:
            if gc_was_on:
                gc.enable()
        te = reduce_max(statistics.median(calls), dist, dev)
        e2e = {"value": n * world / te, "unit": "strings/s", "h2d_bytes_per_step": int(len(s.chars) + 8 * n),
               "d2h_bytes_per_step": int(8 * n), "ms_per_step": te * 1e3,
               "ms_per_step_mean": reduce_max(sum(calls) / len(calls), dist, dev) * 1e3,
               "ms_per_step_max": reduce_max(max(calls), dist, dev) * 1e3, "steps": len(calls),
               "timing": "median of the per-call host times, max over ranks"}
        e2e["link"] = host_link(torch, stream, dev, h_chars, h_perm, chars, perm, e2e, ms)

    legs = set(x for x in args.legs.split(",") if x and x != "none")
    extra = {}
    if "host" in legs:
        extra["host_driven_form"] = leg_host(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world,
                                             dist)
    if "keys8" in legs:
        extra["graph_form_keys8"] = leg_keys8(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world,
                                              dist)
    if "equal" in legs:
        extra["graph_form_equal"] = leg_equal(sss, torch, chars, offsets, perm, lcp, n, stream, dev, args, world,
                                              dist)
    if "learned" in legs:
        extra["learned"] = leg_learned(sss, torch, stream, dev, args, world, dist)
    if "batched" in legs:
        extra["batched"] = leg_batched(sss, torch, stream, dev, args, world, dist)
    if "alphabet" in legs:
        extra["alphabet"] = leg_alphabet(sss, torch, stream, dev, args, world, dist)
    if "uniform" in legs:
        extra["uniform_100k"] = leg_uniform(sss, torch, stream, dev, args, world, dist)
    if "literal" in legs:
        del chars, offsets, perm, lcp
        extra["batched_literal"] = leg_literal(sss, torch, stream, dev, args, world, dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel: k_scatter, the largest share of the
    # serialised launch list (profiles/launches_url-16m.txt) and the last
    # kernel of the device-wide round, whose branch runs at the highest
    # stream priority (the other branches' event times include the time
    # they yield the SMs to it)
    cls = sss.K_CLASSES
    dom = cls.index("scatter") if prof_launches[cls.index("scatter")] else int(np.argmax(prof_ms))
    # algorithmic bytes per kernel class: device-wide rounds (k_classify,
    # k_scatter) see the large segments' strings, k_med_round the medium ones
    algo = {"scatter": SCATTER_BYTES_PER_STRING * large_strings + REFILL_BYTES * large_refills,
            "classify": CLASSIFY_BYTES_PER_STRING * (large_strings - fused_root_strings),
            "medium": MEDIUM_BYTES_PER_STRING * medium_strings + REFILL_BYTES * medium_refills,
            "base": BASE_BYTES_PER_STRING * base_strings}
    units = {"scatter": large_strings, "classify": large_strings - fused_root_strings, "medium": medium_strings,
             "base": base_strings}
    kname = {"scatter": "k_scatter", "classify": "k_classify", "base": "k_base",
             "medium": "k_med_round"}.get(cls[dom], "k_" + cls[dom])
    peak, peak_kind = measured_hbm_peak()
    roofline = None
    if cls[dom] in algo and prof_ms[dom] > 0:
        achieved = algo[cls[dom]] / (prof_ms[dom] * 1e-3) / 1e9
        per_launch_units = units[cls[dom]] / max(1, prof_launches[dom])
        tb = ncu_traffic(kname, args.workload)
        roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_kind": f"of {peak_kind}",
                    "traffic": (tb * per_launch_units if tb is not None else None),
                    "algorithmic_bytes_per_launch": algo[cls[dom]] / max(1, prof_launches[dom]),
                    "avg_launch_ms": prof_ms[dom] / max(1, prof_launches[dom])}
    # distribution-round kernels together (classify + scan + scatter)
    rounds_ms = prof_ms[cls.index("classify")] + prof_ms[cls.index("scatter")] + prof_ms[cls.index("scan")]
    rounds_bytes = algo["scatter"] + algo["classify"]
    kernel_share = {cls[i]: {"ms_per_step": prof_ms[i] / args.steps,
                             "launches_per_step": int(prof_launches[i]) // args.steps}
                    for i in range(len(cls)) if prof_launches[i]}

    cpu = None
    D = None
    if oracle_info and "error" not in oracle_info:
        D = oracle_info["D"]
        cpu = {"value": oracle_info["cpu_n"] / oracle_info["cpu_s"], "unit": "strings/s", "cores": 1,
               "host_cores": oracle_info["cpu_cores"], "kind": "oracle",
               "sample": (f"first {oracle_info['cpu_n']} strings of the {args.workload} workload "
                          f"(same generator and seed), one sort, single thread"),
               "parallel": {"value": oracle_info["cpu_n"] / oracle_info["cpu_par_s"], "unit": "strings/s",
                            "cores": oracle_info["cpu_cores"], "kind": "oracle",
                            "sample": "the same strings, sample-cut ranges sorted on one thread per host core"}}
    value = n * world / (ms * 1e-3)
    line = {
        "metric": "sorted strings/s", "value": value, "unit": "strings/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_mean": ms_mean,
        "timing": "median of the per-step CUDA-event times (each step one sort), max over ranks",
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOAD_TEXT.get(args.workload, ""),
                   "mode": args.mode, "form": "graph", "key_bytes": int(opts.key_bytes), "n": n, "chars_bytes": int(s.total),
                   "D": D, "D_over_N": (D / s.total) if D else None,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}"},
        "d_bytes_per_s": (D * world / (ms * 1e-3)) if D else None,
        "rounds_hbm": {"achieved": rounds_bytes / (rounds_ms * 1e-3) / 1e9 if rounds_ms else None,
                       "peak": peak, "unit": "GB/s",
                       "frac": (rounds_bytes / (rounds_ms * 1e-3) / 1e9 / peak) if rounds_ms else None},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": int(launches[0]),
        "kernels": kernel_share,
        "profiled_pass": {"form": "host-driven rounds, CUDA events around every launch", "steps": args.steps,
                          "ms_per_step": ms_profiled},
        "sort_stats": {k: last_stats[k] for k in ("rounds", "base_tiles", "round_strings", "medium_strings",
                                                  "base_strings", "refilled_strings", "medium_refilled_strings",
                                                  "learned_keys", "learned_misses")},
    }
    line.update(extra)
    if oracle_info and "error" in oracle_info:
        line["oracle_error"] = oracle_info["error"]
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
