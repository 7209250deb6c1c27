"""Benchmark of the longest-overlap-region path on GB300.

One step = the whole path over one synthetic instance: encode + concatenate
(a1), DC3 suffix array (a2-a8), ISA + LCP (a9), longest overlap with all
positions (a10), sparse table (a11) and 1M LCP queries (a12).  The default
workload is two iid-uniform sequences of 134,217,728 bases with one planted
500-base common region (S1#S2$, n = 268,435,458), plus 1,000,000 uniform
(p, q) queries.  ``value`` = input bases per second with inputs resident in
HBM; ``e2e`` repeats it with the ASCII input and queries copied from pinned
host memory and the results copied back inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lor|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator kwargs, queries, description)
    "large": (dict(n_each=134_217_728, seed=140434483), 1_000_000,
              "2x134217728 iid-uniform DNA with one 500-base plant, S1#S2$ (n=268435458); "
              "1M uniform LCP queries"),
    "noncoding": (None, 1_000_000,
                  "2x16777216 noncoding-like DNA (40% GC, repeats, microsatellites, 10 kb shared "
                  "region with exact 2 kb core), S1#S2$; 1M uniform LCP queries"),
    "tiny": (dict(n_each=100_000, seed=140434481), 100_000,
             "2x100000 iid-uniform DNA with one 500-base plant, S1#S2$; 100k LCP queries"),
}
METRIC = "input bases/s for SA+LCP+longest overlap (1 GB300)"
UNIT = "bases/s"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(vals, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity on
    one process).  Used for the timed region: the job is as slow as its
    slowest replica."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(units_per_rank, world, ms):
    """Whole-job units per second: every rank processed units_per_rank in at
    most ms milliseconds."""
    return world * units_per_rank / (ms / 1000.0)


def percentile(vals, q):
    v = sorted(vals)
    if not v:
        return None
    k = min(len(v) - 1, max(0, int(round(q / 100.0 * (len(v) - 1)))))
    return v[k]


def make_inputs(name):
    import lor_inputs as gen
    kw, nq, desc = WORKLOADS[name]
    if name == "noncoding":
        seqs, info = gen.pair_noncoding()
    else:
        seqs, info = gen.pair_uniform(**kw)
    n = sum(len(s) for s in seqs) + len(seqs)
    p, q = gen.random_queries(n, count=nq)
    return seqs, info, p, q, desc


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1404_3448_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


TRAFFIC_PROFILES = {"large": "dram_by_kind_2x134217728.md"}


def ncu_traffic(kind, workload):
    """DRAM bytes per launch of `kind` from the committed ncu summary of this
    workload (profiles/, written by paper_1404_3448_gb300.ncu_summary), only
    when it was taken on the current kernel sources."""
    name = TRAFFIC_PROFILES.get(workload)
    if not name:
        return None
    try:
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(r"source hash: `([0-9a-f]+)`", text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    for line in text.splitlines():
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) == 6 and cells[0] == kind:
            try:
                return float(cells[5])
            except ValueError:
                return None
    return None


# --------------------------------------------------------------------------- CPU (oracle)

def cpu_sample_run(n_each, seed, nq):
    """One pass of the oracle over a bounded sample of the same generator."""
    import lor_inputs as gen
    import oracle
    seqs, _ = gen.pair_uniform(n_each=n_each, plant_len=500, seed=seed)
    t0 = time.perf_counter()
    text, starts, _ = oracle.encode_concat(seqs)
    sa = oracle.suffix_array(text, nthreads=1)
    lcp = oracle.lcp_array(text, sa, nthreads=1)
    oracle.longest_overlap(text, sa, lcp, starts)
    oracle.sparse_table(lcp)
    p, q = gen.random_queries(len(text), count=nq, seed=seed)
    oracle.lcp_pairs(text, p, q)
    return time.perf_counter() - t0, 2 * n_each


def cpu_baseline(budget_s=15.0):
    import oracle
    oracle.build()
    n_each = 1 << 20
    dt, bases = cpu_sample_run(n_each, 140434483, 10_000)
    # scale the sample so it takes roughly the budget, then time it once more
    scale = max(1, min(8, int(budget_s / max(dt, 1e-3))))
    if scale > 1:
        dt, bases = cpu_sample_run(n_each * scale, 140434483, 10_000 * scale)
    return {"value": bases / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"oracle (merge-sort SA, naive LCP, overlap scan, sparse table, direct-"
                      f"comparison queries) on 2x{n_each * scale} iid-uniform bases, 1 thread, "
                      f"{dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    n_each = args.ref_bases // 2
    for i in range(args.warmup):
        cpu_sample_run(n_each, 1000 + i, 20000)
    total_t, total_b = 0.0, 0
    for i in range(args.steps):
        dt, b = cpu_sample_run(n_each, 2000 + i, 20000)
        total_t += dt
        total_b += b
    value = total_b / total_t
    sample = (f"oracle on 2x{n_each} iid-uniform bases per step (encode, merge-sort SA, naive "
              f"LCP, overlap scan, sparse table, 20000 direct-comparison queries), 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][2], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- batched

def batch_vs_plain(npairs, steps, warmup, dev, seed=140434484):
    """The same npairs sequence pairs (per-sequence lengths log-uniform in
    [1k, 1M], noncoding-like) through lor_batch_overlap, and one pair per
    call through encode + SA + LCP + overlap.  Returns a dict of throughputs
    and per-pair latencies of the plain path."""
    import torch
    import lor_inputs as gen
    import paper_1404_3448_gb300 as lor
    from paper_1404_3448_gb300 import lor as C

    pairs = gen.pair_batch(npairs=npairs, seed=seed)
    flat = [x for pr in pairs for x in pr]
    lens = np.array([len(x) for x in flat], dtype=np.int64)
    n_bases = int(lens.sum())
    ascii_dev = torch.from_numpy(np.concatenate(flat)).to(dev)
    stream = torch.cuda.current_stream(dev)

    # launch parameters tuned on the first group's worth of pairs (the
    # autotuner times lor_batch_overlap on them); both batched runs use them
    ns = min(npairs, 512)
    nl = lens[: 2 * ns]
    t0 = time.perf_counter()
    tb = lor.lor.Batch(nl, device=dev, pos_cap=1 << 22)
    lor.tune_set(**lor.tune_default())
    tuned, tuned_ms = lor.autotune_batch(tb, ascii_dev[: int(nl.sum())], reps=2)
    tune_s = time.perf_counter() - t0
    del tb
    torch.cuda.empty_cache()

    b = lor.lor.Batch(lens, device=dev, pos_cap=1 << 24)
    for _ in range(warmup):
        b.run(ascii_dev)
    torch.cuda.synchronize(dev)
    lor.check_device(where="batch warmup")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for i in range(steps):
        b.run(ascii_dev)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    batch_ms = evs[0].elapsed_time(evs[-1]) / steps
    batch_steps = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
    eager_out = b.out.clone()
    del b
    torch.cuda.empty_cache()

    # the same pipeline captured once into a CUDA graph and replayed
    t0 = time.perf_counter()
    gb = lor.lor.BatchGraph(lens, ascii_dev, device=dev, pos_cap=1 << 24)
    capture_s = time.perf_counter() - t0
    for _ in range(warmup):
        gb.run()
    torch.cuda.synchronize(dev)
    lor.check_device(where="batch graph warmup")
    graph_same = bool(torch.equal(gb.out, eager_out))
    gev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    gev[0].record(stream)
    for i in range(steps):
        gb.run()
        gev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    graph_ms = gev[0].elapsed_time(gev[-1]) / steps
    graph_steps = [gev[i].elapsed_time(gev[i + 1]) for i in range(steps)]
    graph_kernels = gb.kernels
    gb.close()
    del gb
    torch.cuda.empty_cache()

    # plain: one pair per call, buffers sized for the largest pair
    nmax = int(max(lens[0::2] + lens[1::2])) + 2
    text = torch.empty(nmax, dtype=torch.uint8, device=dev)
    starts = torch.empty(3, dtype=torch.int32, device=dev)
    sa = torch.empty(nmax, dtype=torch.int32, device=dev)
    isa = torch.empty(nmax, dtype=torch.int32, device=dev)
    lcp = torch.empty(nmax, dtype=torch.int32, device=dev)
    out = torch.empty(8, dtype=torch.int32, device=dev)
    pos = torch.empty(1 << 20, dtype=torch.int32, device=dev)
    ws = lor.workspace(max(C.lor_build_sa_workspace_size(nmax, 7), C.lor_lcp_workspace_size(nmax),
                           C.lor_longest_overlap_workspace_size(nmax)), dev)
    offs = np.concatenate([[0], np.cumsum(lens)])
    s = int(stream.cuda_stream)

    def plain_pair(p):
        l2 = lens[2 * p:2 * p + 2].copy()
        n = int(l2.sum()) + 2
        a = ascii_dev[int(offs[2 * p]):int(offs[2 * p + 2])]
        C._check(C.lor_encode_concat(a.data_ptr() if a.numel() else None, l2.ctypes.data, 2,
                                     text.data_ptr(), starts.data_ptr(), s), "encode")
        C._check(C.lor_build_sa(text.data_ptr(), n, 7, sa.data_ptr(), ws.data_ptr(), ws.numel(), s),
                 "build_sa")
        C._check(C.lor_lcp(text.data_ptr(), sa.data_ptr(), n, isa.data_ptr(), lcp.data_ptr(),
                           ws.data_ptr(), ws.numel(), s), "lcp")
        C._check(C.lor_longest_overlap(sa.data_ptr(), lcp.data_ptr(), n, starts.data_ptr(), 2,
                                       out.data_ptr(), pos.data_ptr(), pos.numel(), ws.data_ptr(),
                                       ws.numel(), s), "overlap")

    for p in range(min(npairs, 16)):
        plain_pair(p)
    torch.cuda.synchronize(dev)
    pe = [torch.cuda.Event(enable_timing=True) for _ in range(npairs + 1)]
    pe[0].record(stream)
    for p in range(npairs):
        plain_pair(p)
        pe[p + 1].record(stream)
    torch.cuda.synchronize(dev)
    lor.check_device(where="plain pairs")
    plain_ms = pe[0].elapsed_time(pe[-1])
    per_pair = [pe[i].elapsed_time(pe[i + 1]) for i in range(npairs)]
    batch_value = n_bases / (batch_ms / 1000.0)
    graph_value = n_bases / (graph_ms / 1000.0)
    plain_value = n_bases / (plain_ms / 1000.0)
    return {
        "workload": f"{npairs} noncoding-like pairs, per-sequence lengths log-uniform in [1k, 1M], "
                    f"one shared plant of 50-5000 bases per pair ({n_bases} bases)",
        "pairs": npairs, "input_bases": n_bases,
        "batched": {"value": batch_value, "unit": UNIT, "ms_per_step": batch_ms,
                    "step_latency_ms": {"p50": percentile(batch_steps, 50),
                                        "p99": percentile(batch_steps, 99)}, "steps": steps},
        "batched_graph": {"value": graph_value, "unit": UNIT, "ms_per_step": graph_ms,
                          "step_latency_ms": {"p50": percentile(graph_steps, 50),
                                              "p99": percentile(graph_steps, 99)}, "steps": steps,
                          "capture_s": capture_s, "kernels_per_replay": graph_kernels,
                          "records_equal_eager": graph_same},
        "plain": {"value": plain_value, "unit": UNIT, "ms_all_pairs": plain_ms,
                  "pair_latency_ms": {"p50": percentile(per_pair, 50), "p99": percentile(per_pair, 99),
                                      "max": max(per_pair)}},
        "batched_over_plain": batch_value / plain_value,
        "graph_over_plain": graph_value / plain_value,
        "autotune": {"config": tuned, "default": lor.tune_default(), "sample_pairs": ns,
                     "sample_ms": tuned_ms, "seconds": tune_s},
    }


# --------------------------------------------------------------------------- multi-query

def multi_query_run(nq, steps, warmup, dev, ref_len=1 << 24, seed=140434487):
    """One noncoding-like reference of ref_len bases against nq queries
    (log-uniform lengths in [100, 10,000]; half reads of the reference with
    substitutions) through lor_multi_query_overlap: one suffix array over the
    reference and all queries."""
    import torch
    import lor_inputs as gen
    import paper_1404_3448_gb300 as lor
    ref, qs = gen.multi_query(ref_len=ref_len, nq=nq, seed=seed)
    lens = [len(q) for q in qs]
    qbases = int(sum(lens))
    ref_dev = torch.from_numpy(ref).to(dev)
    q_dev = torch.from_numpy(np.concatenate(qs)).to(dev)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((nq, 4), dtype=torch.int32, device=dev)
    need = lor.lor.load().lor_multi_query_workspace_size(ref.size, np.asarray(lens, np.int64).ctypes.data, nq)
    ws = lor.workspace(need, dev)
    for _ in range(warmup):
        lor.multi_query_overlap(ref_dev, q_dev, lens, out=out, ws=ws)
    torch.cuda.synchronize(dev)
    lor.check_device(where="multi query warmup")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for i in range(steps):
        lor.multi_query_overlap(ref_dev, q_dev, lens, out=out, ws=ws)
        evs[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    ms = evs[0].elapsed_time(evs[-1]) / steps
    found = out[:, 0].cpu().numpy()
    del ws
    torch.cuda.empty_cache()
    return {
        "workload": f"one {ref_len}-base noncoding-like reference against {nq} queries (log-uniform lengths "
                    f"in [100, 10000], half reads of the reference with 1-5 % substitutions, half background "
                    f"with one planted 20-200-base piece); {qbases} query bases",
        "queries": nq, "query_bases": qbases, "ms_per_step": ms,
        "value": (qbases + ref_len) / (ms / 1000.0), "unit": UNIT,
        "queries_per_s": nq / (ms / 1000.0),
        "median_match_length": float(np.median(found)),
    }


# --------------------------------------------------------------------------- 64-bit indices

def int64_run(n_each, steps, warmup, dev):
    """The 64-bit index path (lor_encode_concat64 once, then per step
    lor_build_sa64, lor_lcp64 and lor_longest_overlap64) on two uniform
    sequences whose concatenation passes 2^31 symbols.  One workspace serves
    the suffix array and the LCP call (they run one after the other)."""
    import torch
    import lor_inputs as gen
    import paper_1404_3448_gb300 as lor
    C = lor.lor.load()
    seqs, info = gen.pair_int64(n_each=n_each)
    lens = [len(x) for x in seqs]
    ascii_dev = torch.from_numpy(np.concatenate(seqs)).to(dev)
    del seqs
    text, starts, sigma = lor.encode_concat64(ascii_dev, lens)
    del ascii_dev
    n = text.numel()
    need = max(C.lor_build_sa64_workspace_size(n, sigma), C.lor_lcp64_workspace_size(n),
               C.lor_longest_overlap64_workspace_size(n))
    ws = lor.workspace(need, dev)
    sa = torch.empty(n, dtype=torch.int64, device=dev)
    isa = torch.empty(n, dtype=torch.int64, device=dev)
    lcp = torch.empty(n, dtype=torch.int32, device=dev)
    out = torch.empty(48, dtype=torch.uint8, device=dev)
    pos = torch.empty(1 << 16, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        lor.build_sa64(text, sigma, sa=sa, ws=ws)
        if evs:
            evs[1].record(stream)
        lor.lcp64(text, sa, isa=isa, lcp_out=lcp, ws=ws)
        if evs:
            evs[2].record(stream)
        lor.longest_overlap64(sa, lcp, starts, 2, pos_cap=pos.numel(), out=out, pos=pos, ws=ws)
        if evs:
            evs[3].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    lor.check_device(where="int64 warmup")
    parts = np.zeros(3)
    for _ in range(steps):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        step(evs)
        torch.cuda.synchronize(dev)
        parts += [evs[i].elapsed_time(evs[i + 1]) for i in range(3)]
    lor.check_device(where="int64 steps")
    parts /= steps
    ms = float(parts.sum())
    rec = lor.overlap64_dict(out, pos)
    del ws, sa, isa, lcp, text
    torch.cuda.empty_cache()
    return {
        "workload": f"2x{n_each} iid-uniform DNA (n={n}, past 2^31) with one 500-base plant, the copy in the "
                    f"second sequence past text position 2^31; int64 SA/ISA, int32 LCP",
        "n": n, "input_bases": int(sum(lens)), "steps": steps, "ms_per_step": ms,
        "value": sum(lens) / (ms / 1000.0), "unit": UNIT,
        "stage_ms": {"build_sa64": float(parts[0]), "lcp64": float(parts[1]), "overlap64": float(parts[2])},
        "overlap": {"length": int(rec["length"]), "n_pos": int(rec["n_pos"])},
    }


# --------------------------------------------------------------------------- served

def serving(seconds, rate, pool_pairs, workers, budget_gb, dev, queries=16, seed=140434485):
    """Requests arrive as a Poisson process (``rate`` per second for
    ``seconds``), each asking for one pair of a pool of noncoding-like pairs
    (per-sequence lengths log-uniform in [1k, 4M]) held in pinned host memory.
    A submitter thread submits on the arrival clock to a lor_server with a
    ``budget_gb`` device reservation; the main thread polls results, asks the
    request's ``queries`` follow-up LCP queries on its resident state and
    releases it.  Reports sustained input bases/s and latency percentiles."""
    import threading
    import torch
    import lor_inputs as gen
    import paper_1404_3448_gb300 as lor

    pool = gen.pair_batch(npairs=pool_pairs, lo=1_000, hi=4_000_000, seed=seed)
    lens = [(len(a), len(b)) for a, b in pool]
    total = sum(a + b for a, b in lens)
    host = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    hv = host.numpy()
    ptrs, off = [], 0
    for a, b in pool:
        hv[off:off + len(a)] = a
        hv[off + len(a):off + len(a) + len(b)] = b
        ptrs.append((host.data_ptr() + off, host.data_ptr() + off + len(a)))
        off += len(a) + len(b)
    arrivals = gen.poisson_arrivals(rate, seconds, seed=seed + 1)
    choice, P, Q = gen.request_stream(len(arrivals), lens, queries=queries, seed=seed + 2)
    nreq = len(arrivals)

    srv = lor.Server(int(budget_gb * (1 << 30)), workers=workers, max_batch_pairs=512)
    try:
        # warm-up: every pool pair once, so first-launch setup is not timed
        for k in range(pool_pairs):
            srv.submit_ptr(ptrs[k][0], lens[k][0], ptrs[k][1], lens[k][1], tag=k)
        got = 0
        while got < pool_pairs:
            for r in srv.poll(timeout_ms=100):
                if r["status"] != 0:
                    raise RuntimeError(f"warm-up request failed: {lor.lor.status_string(r['status'])}")
                srv.release(r["id"])
                got += 1
        first = {}
        lat, qlat, sub_t, done_t = [], [], [], []
        errors = []
        t0 = srv.now() + 0.05

        def submitter():
            try:
                for k in range(nreq):
                    while True:
                        wait = t0 + arrivals[k] - srv.now()
                        if wait <= 0:
                            break
                        time.sleep(min(wait, 0.001))
                    c = int(choice[k])
                    srv.submit_ptr(ptrs[c][0], lens[c][0], ptrs[c][1], lens[c][1], tag=k)
            except Exception as e:  # surfaced by the main thread
                errors.append(e)

        th = threading.Thread(target=submitter, daemon=True)
        th.start()
        done = 0
        consistent = True
        while done < nreq and not errors:
            for r in srv.poll(timeout_ms=20):
                k = int(r["tag"])
                if r["status"] != 0:
                    raise RuntimeError(f"request {k} failed: {lor.lor.status_string(r['status'])}")
                q0 = time.perf_counter()
                ans = srv.query(r["id"], P[k], Q[k])
                qlat.append((time.perf_counter() - q0) * 1000.0)
                c = int(choice[k])
                rec = (r["length"], r["rank"], r["pos_a"], r["pos_b"], r["n_pos"])
                if first.setdefault(c, rec) != rec:
                    consistent = False
                if ans.min() < 0:
                    consistent = False
                srv.release(r["id"])
                lat.append((r["t_done"] - r["t_submit"]) * 1000.0)
                sub_t.append(r["t_submit"])
                done_t.append(r["t_done"])
                done += 1
        th.join()
        if errors:
            raise errors[0]
        st = srv.stats()
    finally:
        srv.close()
    bases = int(sum(lens[int(c)][0] + lens[int(c)][1] for c in choice))
    span = max(done_t) - min(sub_t)
    return {
        "workload": f"Poisson arrivals at {rate:g} pair requests/s for {seconds:g} s; pairs drawn uniformly "
                    f"from a pool of {pool_pairs} noncoding-like pairs (per-sequence lengths log-uniform in "
                    f"[1k, 4M]) in pinned host memory; {queries} follow-up LCP queries per pair on resident "
                    f"state; {budget_gb:g} GB device budget; {workers} workers",
        "requests": nreq, "input_bases": bases,
        "offered_bases_per_s": bases / float(arrivals[-1]) if nreq else 0.0,
        "value": bases / span, "unit": UNIT,
        "latency_ms": {"p50": percentile(lat, 50), "p99": percentile(lat, 99), "max": max(lat)},
        "query_call_ms": {"p50": percentile(qlat, 50), "p99": percentile(qlat, 99)},
        "batches": st["batches"], "mean_batch_pairs": st["pairs"] / max(st["batches"], 1),
        "admission_waits": st["admission_waits"], "peak_reserved_gb": st["peak_bytes"] / 2**30,
        "results_consistent": consistent,
    }


# --------------------------------------------------------------------------- GPU

def run_lor(args):
    import torch
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3448_gb300 as lor
    from paper_1404_3448_gb300 import lor as C

    seqs, info, p_np, q_np, desc = make_inputs(args.workload)
    lens = [len(s) for s in seqs]
    n_bases = int(sum(lens))
    host_ascii = torch.from_numpy(np.concatenate(seqs)).pin_memory()
    host_p = torch.from_numpy(p_np).pin_memory()
    host_q = torch.from_numpy(q_np).pin_memory()
    ascii_dev = host_ascii.to(dev)
    p_dev, q_dev = host_p.to(dev), host_q.to(dev)
    ans_dev = torch.empty_like(p_dev)
    pipe = lor.Pipeline(lens, device=dev, pos_cap=1 << 16)
    host_out = torch.empty(8, dtype=torch.int32).pin_memory()
    host_pos = torch.empty(1 << 16, dtype=torch.int32).pin_memory()
    host_ans = torch.empty_like(host_p).pin_memory()
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step():
        pipe.run(ascii_dev, p_dev, q_dev, ans_dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    lor.check_device(where="warmup")

    # ---- device-resident timed region
    lor.profile_reset()
    lor.profile_enable(True)
    launches0 = C.lor_launch_count()
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize(dev)
    barrier()
    launches = C.lor_launch_count() - launches0
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    ms = evs[0].elapsed_time(evs[-1]) / args.steps
    prof = lor.profile_read()
    lor.profile_enable(False)
    lor.check_device(where="timed")

    # ---- end to end: pinned host in, results back to host
    torch.cuda.synchronize(dev)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    npos = 0
    for _ in range(args.steps):
        ascii_dev.copy_(host_ascii, non_blocking=True)
        p_dev.copy_(host_p, non_blocking=True)
        q_dev.copy_(host_q, non_blocking=True)
        out, pos = pipe.run(ascii_dev, p_dev, q_dev, ans_dev)
        host_out.copy_(out, non_blocking=True)
        host_ans.copy_(ans_dev, non_blocking=True)
        stream.synchronize()
        npos = min(int(host_out[6]), pos.numel())
        if npos:
            host_pos[:npos].copy_(pos[:npos], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / args.steps

    # ---- linear-space RMQ on the same LCP array and queries (a side measurement)
    rmq_linear = None
    try:
        btab = lor.rmq_block_build(pipe.lcp)
        bans = torch.empty_like(p_dev)
        torch.cuda.synchronize(dev)
        r0, r1, r2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        reps = 5
        r0.record(stream)
        for _ in range(reps):
            lor.rmq_block_build(pipe.lcp, table=btab)
        r1.record(stream)
        for _ in range(reps):
            lor.rmq_block_query(btab, pipe.lcp, pipe.isa, p_dev, q_dev, out=bans)
        r2.record(stream)
        torch.cuda.synchronize(dev)
        lor.check_device(where="block rmq")
        pipe.run(ascii_dev, p_dev, q_dev, ans_dev)
        torch.cuda.synchronize(dev)
        rmq_linear = {
            "table_bytes": int(btab.numel()) * 4,
            "sparse_table_bytes": int(pipe.table.numel()) * 4,
            "build_ms": r0.elapsed_time(r1) / reps,
            "query_ms": r1.elapsed_time(r2) / reps,
            "queries": int(p_np.size),
            "answers_equal_sparse_table": bool(torch.equal(bans, ans_dev)),
        }
        del btab, bans
    except Exception as exc:  # reported, not hidden
        rmq_linear = {"error": str(exc)}

    ms_all, e2e_all, p50, p99 = max_over_ranks(
        [ms, e2e_ms, percentile(step_ms, 50), percentile(step_ms, 99)], device=dev)

    if rank == 0:
        value = job_throughput(n_bases, world, ms_all)
        e2e_value = job_throughput(n_bases, world, e2e_all)
        h2d = host_ascii.numel() + 4 * (host_p.numel() + host_q.numel())
        d2h = 32 + 4 * host_ans.numel() + 4 * npos
        stage_ms = {k: v["ms"] / args.steps for k, v in prof.items()}
        dom = max(prof, key=lambda k: prof[k]["ms"]) if prof else None
        peak, peak_src = measured_peak_gbs()
        roof = None
        if dom:
            d = prof[dom]
            achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9
            roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                    "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src,
                    "launches_per_step": d["launches"] / args.steps,
                    "algorithmic_bytes_per_launch": d["bytes"] / d["launches"],
                    "avg_launch_ms": d["ms"] / d["launches"],
                    "traffic": ncu_traffic(dom, args.workload)}
        path_bytes = sum(v["bytes"] for v in prof.values()) / args.steps
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_all,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "n": pipe.n, "input_bases": n_bases,
                       "queries": int(p_np.size), "parallelism": "replicas" if world > 1 else "none",
                       "l2": "inputs larger than L2 (268 MB text, >10 GB working set)",
                       "step": "a1-a12: encode, DC3 SA, ISA+LCP, overlap+positions, sparse "
                               "table, LCP queries"},
            "roofline": roof,
            "path_model_bytes_per_step": path_bytes,
            "path_model_gbs": path_bytes / (ms / 1000.0) / 1e9,
            "stage_ms": stage_ms,
            "step_latency_ms": {"p50": p50, "p99": p99, "mean": ms_all, "steps": args.steps},
            "overlap": {"length": int(host_out[0]), "n_pos": int(host_out[6])},
            "dc3_levels": len(lor.last_dc3_trace()),
            "clocks": clocks.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "rmq_linear": rmq_linear,
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        if args.batch_pairs > 0:
            del pipe
            torch.cuda.empty_cache()
            line["batch_vs_plain"] = batch_vs_plain(args.batch_pairs, 3, 1, dev)
        if args.multi_queries > 0:
            torch.cuda.empty_cache()
            line["multi_query"] = multi_query_run(args.multi_queries, 3, 1, dev)
        if args.int64_bases > 0:
            torch.cuda.empty_cache()
            line["int64"] = int64_run(args.int64_bases // 2, 2, 1, dev)
        if args.serve_seconds > 0:
            torch.cuda.empty_cache()
            line["serving"] = serving(args.serve_seconds, args.serve_rate, args.serve_pool, args.serve_workers,
                                      args.serve_budget_gb, dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lor", choices=["lor", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-pairs", type=int, default=4096,
                    help="pairs of the batched-vs-plain sub-measurement (0 skips it)")
    ap.add_argument("--multi-queries", type=int, default=65_536,
                    help="queries of the one-reference-many-queries sub-measurement (0 skips it)")
    ap.add_argument("--int64-bases", type=int, default=2 * ((1 << 30) + (1 << 15)),
                    help="input bases of the 64-bit index sub-measurement (past 2^31 symbols; 0 skips it)")
    ap.add_argument("--serve-seconds", type=float, default=3.0,
                    help="seconds of Poisson arrivals of the served sub-measurement (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="pair requests per second")
    ap.add_argument("--serve-pool", type=int, default=256, help="distinct pairs the requests draw from")
    ap.add_argument("--serve-workers", type=int, default=2)
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    ap.add_argument("--ref-bases", type=int, default=1 << 22,
                    help="bases per step of the reference (oracle) arm")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_lor(args)


if __name__ == "__main__":
    sys.exit(main())
