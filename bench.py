"""Benchmark of the IVF-PQ filtering path on one B300 (or N replicas).

Workload (default): 10M uint8 d=128 vectors from a 64-component Gaussian
mixture clipped to 0..255 (SIFT-like, the paper's Table 1 shape), 16384 lists,
PQ M=32 x 256, 10k queries, k 10. Operating point (default): nprobe 144 and an
exhaustive Algorithm 1 re-rank (eps < 0) of the ADC top-12288 on raw rows held
in HBM, the fastest measured point whose recall@10 is safely above 0.9 (the
configured nprobe 64 with a re-rank of the top 10k = 100 reaches 0.18 on this
data). ``value`` is the precision form (BF16 tensor-core probe and LUT, FP16
table); the plain FP32 form runs on the same index and point beside it.
recall@10 is measured on a 1k-query subsample in every run; ``--sweep`` prints
the recall/QPS curve over nprobe, n and Algorithm 1's parameters.

A step is one batch of 10k queries through the whole path: coarse probe, LUT,
gather + dedup, ADC scan + top-n, re-rank. ``value`` is queries per second
with the queries already in HBM; ``e2e`` is the same through the C ABI with
host buffers (host->device copy of the queries and device->host copy of the
results inside the timed region). ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

L2_BYTES = 126 * 1024 * 1024
NOMINAL_HBM_GBS = 7700.0  # B300 HBM3e nominal; the measured copy bandwidth is the roofline peak
SCAN_SOURCES = ["paper_2409_16576_b300/csrc/kernels/k_scan.cu",
                "paper_2409_16576_b300/csrc/kernels/warp_topk.cuh",
                "paper_2409_16576_b300/csrc/kernels/rerank_rows.cuh"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--form", default="lowp", choices=["lowp", "plain", "batched"],
                    help="lowp: BF16 tensor-core probe and LUT, FP16 LUT (precision form); batched: the "
                         "same table scanned list by list over the whole batch (FA_BATCHED); plain: FP32 "
                         "everywhere; all re-rank the ADC top-n")
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--nq", type=int, default=10_000)
    # default operating point: the fastest measured (nprobe, re-rank depth) with
    # recall@10 safely above 0.9 on this workload (0.910 on the 1k-query
    # subsample; nprobe 64 with n = 10 k = 100, the configured point, reaches 0.18)
    ap.add_argument("--nprobe", type=int, default=144)
    ap.add_argument("--rerank-n", type=int, default=12288, help="re-rank the ADC top-n")
    ap.add_argument("--batch", type=int, default=32, help="Algorithm 1 BatchSize")
    ap.add_argument("--eps", type=float, default=-1.0, help="Algorithm 1 epsilon (< 0: no early stop)")
    ap.add_argument("--beta", type=int, default=1, help="Algorithm 1 beta")
    ap.add_argument("--raw", default="device", choices=["device", "host"],
                    help="raw vectors for the re-rank: HBM or pinned host memory")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip timing the plain FP32 form at the same operating point")
    ap.add_argument("--no-batching", action="store_true",
                    help="skip the batching form's recall-0.9 point (10M Zipf lists, top-100 re-rank)")
    ap.add_argument("--persistent", action="store_true")
    ap.add_argument("--lut", default="fp16", choices=["fp16", "fp8"], help="LUT storage (lowp form)")
    ap.add_argument("--cpu-sample", type=int, default=0, help="queries in the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--recall", type=int, default=1000, help="queries in the recall subsample (0 = off)")
    ap.add_argument("--sweep", action="store_true", help="recall/QPS grid instead of one bench line")
    ap.add_argument("--points", default="",
                    help="sweep points form:nprobe:n:batch:eps:beta, comma-separated (default grid if empty)")
    ap.add_argument("--kmeans-iters", type=int, default=25, help="k-means iterations of the index build")
    ap.add_argument("--serial", action="store_true",
                    help="re-rank after the whole scan (FA_SERIAL) instead of the pipelined chunks")
    ap.add_argument("--spacev-n", type=int, default=10_000_000)
    ap.add_argument("--spacev-M", type=int, default=25, choices=[20, 25, 50])
    ap.add_argument("--metric", default="ip", choices=["ip", "l2"], help="spacev workload: search metric")
    ap.add_argument("--workload", default="sift10m", choices=["sift10m", "zipf", "billion", "spacev"],
                    help="zipf: the batching-form workload (Zipf lists, per-query nprobe); billion: the "
                         "billion-scale shape (4096-component uint8 mixture, 262144 lists, Eq. 2 "
                         "replication) at --billion-n vectors")
    ap.add_argument("--billion-n", type=int, default=250_000_000)
    ap.add_argument("--billion-graph", default="32:4096",
                    help="billion workload: R:S of the navigation graph of the lists (none: no graph probe)")
    ap.add_argument("--graph-points", default="32:8192:8:64:600,48:8192:8:64:700,64:8192:8:64:700,"
                                              "64:8192:16:128:2000",
                    help="billion workload: nprobe:rerank_n:entry:beam:max_check points of the graph probe")
    ap.add_argument("--billion-points", default="32:8192,48:8192,64:8192,128:8192",
                    help="nprobe:rerank_n operating points of the billion workload")
    ap.add_argument("--repl", type=float, default=1.08,
                    help="billion workload: mean lists per vector of Eq. 2's replication")
    ap.add_argument("--zipf-n", type=int, default=100_000_000)
    ap.add_argument("--zipf-rerank", type=int, default=0,
                    help="batching form: re-rank the ADC top-n exhaustively on raw rows in HBM (0 = off)")
    ap.add_argument("--batching-n", type=int, default=100_000_000,
                    help="base size of the batching form's workload in the default line")
    ap.add_argument("--no-tiers", action="store_true",
                    help="skip the re-rank from pinned host rows and from §4.3 pages")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving form (request loop under Poisson load) on the batching index")
    ap.add_argument("--zipf-form", default="batched", choices=["tiled", "batched"],
                    help="batching form's scan: tiled persistent per-query scan (FP8 table) or the "
                         "list-major batched scan (FA_BATCHED, FP16 table)")
    ap.add_argument("--serve", action="store_true",
                    help="serving form: open-loop Poisson arrivals on the Zipf-lists index")
    ap.add_argument("--rates", default="5000,10000,20000,40000,80000")
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--window-us", type=int, default=500)
    ap.add_argument("--serve-form", choices=["tiled", "plain"], default="tiled",
                    help="scan form of the served batches: tiled persistent (uneven work) or one CTA per query")
    return ap.parse_args()


def workload(args):
    w = synth.sift_like_10m()
    return dict(name=w.name if args.n == w.n else "ivfpq-u8-%d-d128-nlist16384-M32" % args.n,
                mix=w.mix, n=args.n, nq=args.nq, nlist=w.nlist, M=w.M, nprobe=args.nprobe, k=w.k,
                rerank_n=args.rerank_n, batch=args.batch,
                eps=args.eps, beta=args.beta, lut=args.lut)


def max_over_ranks(x: float, world: int, device: str) -> float:
    """The largest x over all ranks: the job takes as long as its slowest
    replica (x itself on one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_queries(rank: int, nq: int) -> tuple[int, int]:
    """Query rows of one replica: every rank searches its own batch of nq
    queries against its own copy of the index (weak scaling, no exchange)."""
    return rank * nq, nq


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def src_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_hash, workload):
    """DRAM bytes per scan launch recorded by an ncu capture of this exact
    kernel source on this exact workload (profiles/*.md carries
    'traffic_bytes_per_launch: N', 'kernel_src_hash: H' and
    'traffic_workload: W'), or None."""
    d = os.path.join(ROOT, "profiles")
    if not os.path.isdir(d):
        return None
    for fn in sorted(os.listdir(d)):
        if not fn.endswith(".md"):
            continue
        txt = open(os.path.join(d, fn)).read()
        mh = re.search(r"kernel_src_hash:\s*([0-9a-f]+)", txt)
        mt = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
        mw = re.search(r"traffic_workload:\s*(\S+)", txt)
        if mh and mt and mw and mh.group(1) == kernel_hash and mw.group(1) == workload:
            return float(mt.group(1))
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return j.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_sample(wl, base, queries, parts, nsample):
    """The FP64 oracle (as it stands) on the first nsample queries, all host
    cores; returns (seconds, cores, ids)."""
    import oracle
    off, ids = oracle.lists_from_parts(parts["primary"], parts["rep_off"], parts["rep_ids"],
                                       parts["nlist"])
    cores = cpu_cores()
    oracle.set_threads(cores)
    q = queries[:nsample]
    t0 = time.perf_counter()
    oi, od = oracle.search(q, parts["centroids"], parts["codebooks"], parts["codes"], off, ids,
                           wl["nprobe"], wl["k"], raw=base, rerank_n=wl["rerank_n"],
                           batch=wl["batch"], eps=wl["eps"], beta=wl["beta"])
    return time.perf_counter() - t0, cores, oi


def ground_truth(base, q, k):
    """Brute-force k-NN by exact squared L2 in FP64 on the GPU (exact for
    uint8 data), block by block with a running top-k."""
    import torch
    qs = torch.as_tensor(q, device="cuda", dtype=torch.float64)
    qn = (qs * qs).sum(1, keepdim=True)
    best_d = torch.full((q.shape[0], k), float("inf"), dtype=torch.float64, device="cuda")
    best_i = torch.full((q.shape[0], k), -1, dtype=torch.int64, device="cuda")
    blk = 1 << 18
    for s0 in range(0, base.shape[0], blk):
        x = torch.as_tensor(base[s0:s0 + blk], device="cuda").to(torch.float64)
        dd = qn - 2.0 * (qs @ x.T) + (x * x).sum(1)[None]
        v, i = torch.topk(dd, min(k, x.shape[0]), dim=1, largest=False)
        cd = torch.cat([best_d, v], 1)
        ci = torch.cat([best_i, i + s0], 1)
        o = torch.topk(cd, k, dim=1, largest=False).indices
        best_d, best_i = torch.gather(cd, 1, o), torch.gather(ci, 1, o)
    return best_i.cpu().numpy(), best_d.cpu().numpy()


def ground_truth_u8(base, q, k, ip=False):
    """Brute-force k-NN for uint8 / int8 data with FP32 matrix products (TF32
    off): every dot product, norm and distance is an integer below 2^24, so
    the FP32 results are exact. ip: by the smallest -<q, x>."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        qs = torch.as_tensor(q, device="cuda", dtype=torch.float32)
        qn = torch.zeros((qs.shape[0], 1), device="cuda") if ip else (qs * qs).sum(1, keepdim=True)
        best_d = torch.full((q.shape[0], k), float("inf"), dtype=torch.float32, device="cuda")
        best_i = torch.full((q.shape[0], k), -1, dtype=torch.int64, device="cuda")
        blk = 1 << 22
        for s0 in range(0, base.shape[0], blk):
            x = torch.as_tensor(base[s0:s0 + blk], device="cuda").to(torch.float32)
            dd = -(qs @ x.T) if ip else qn - 2.0 * (qs @ x.T) + (x * x).sum(1)[None]
            v, i = torch.topk(dd, min(k, x.shape[0]), dim=1, largest=False)
            cd = torch.cat([best_d, v], 1)
            ci = torch.cat([best_i, i + s0], 1)
            o = torch.topk(cd, k, dim=1, largest=False).indices
            best_d, best_i = torch.gather(cd, 1, o), torch.gather(ci, 1, o)
        return best_i.cpu().numpy(), best_d.double().cpu().numpy()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def bench_billion(args):
    """The billion-scale shape at args.billion_n vectors: uint8 d=128 from a
    4096-component mixture, 262144 lists by two-level k-means, Eq. 2 boundary
    replication at args.repl lists per vector (the probe-set dedup removes the
    replicas), PQ M=32 codes in HBM, raw rows for the re-rank in HBM (or
    pinned host memory with --raw host), 10k queries. The precision form
    (BF16 tensor-core probe and LUT, FP16 table, per-query scan) is timed at
    each operating point of args.billion_points; the line reports the fastest
    one whose recall@10 on the 1k-query subsample reaches 0.9."""
    import torch
    import oracle
    import paper_2409_16576_b300 as fa
    torch.cuda.set_device(0)
    w = synth.billion_like(args.billion_n)
    nq, k = w.nq, 10
    t0 = time.perf_counter()
    base = w.mix.base(w.n)
    queries = w.mix.queries(nq)
    t_gen = time.perf_counter() - t0
    raw_loc = fa.FA_RAW_DEVICE if args.raw == "device" else fa.FA_RAW_HOST_PINNED
    bp = fa.build_params(nlist=w.nlist, M=w.M, kmeans_iters=min(args.kmeans_iters, 8),
                         repl_eps=-float(args.repl), max_lists_per_vec=8, raw_location=raw_loc)
    t0 = time.perf_counter()
    ix = fa.fa_build_index(base, bp)
    t_build = time.perf_counter() - t0
    info = ix.info()
    ns = min(args.recall or 1000, nq)
    t0 = time.perf_counter()
    gt = ground_truth_u8(base, queries[:ns], 10)
    t_gt = time.perf_counter() - t0
    qd = torch.as_tensor(queries, device="cuda")
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    def point(npb, n, graph=None):
        wl = dict(rerank_n=n, batch=32, eps=-1.0, beta=1, lut="fp16")
        sp = search_params(fa, "lowp", wl)
        if graph:
            sp.probe_gemm = fa.FA_PROBE_GRAPH
            sp.graph_entry, sp.graph_beam, sp.graph_max_check = graph
        _, _, st = fa.fa_search_ex(ix, queries[:1000], k, npb, sp, stats=True)
        ms, tr = timed_steps(fa, torch, ix, qd, k, npb, sp, max(3, min(args.steps, 5)), 3, flush, oid, odist)
        rec = recall_of(oracle, base, queries, oid.cpu().numpy(), gt)
        p = {"probe": "graph" if graph else "exact", "nprobe": npb, "rerank_n": n,
             "qps": nq / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms), "recall_at_10": rec,
             "gathered_per_query": float(st[:, 0].mean()), "distinct_per_query": float(st[:, 1].mean()),
             "stage_ms": {"coarse": statistics.mean(t.coarse_ms for t in tr),
                          "lut": statistics.mean(t.lut_ms for t in tr),
                          "scan": statistics.mean(t.scan_ms for t in tr),
                          "post": statistics.mean(t.post_ms for t in tr)}}
        if graph:
            p.update(entry=graph[0], beam=graph[1], max_check=graph[2])
        print(json.dumps(p), flush=True)
        return p

    points = [point(*(int(x) for x in pt.split(":"))) for pt in args.billion_points.split(",")]
    graph_info = None
    if args.billion_graph != "none":
        # the navigation-graph probe (§4.1) against the exact one, same index
        R, S = (int(x) for x in args.billion_graph.split(":"))
        t0 = time.perf_counter()
        fa.fa_build_probe_graph(ix, R, S)
        graph_info = {"R": R, "S": S, "build_s": time.perf_counter() - t0}
        for pt in args.graph_points.split(","):
            npb, n, e, b, mc = (int(x) for x in pt.split(":"))
            points.append(point(npb, n, (e, b, mc)))
    ok = [p for p in points if p["recall_at_10"] is not None and p["recall_at_10"] >= 0.9]
    best = max(ok, key=lambda p: p["qps"]) if ok else max(points, key=lambda p: p["recall_at_10"] or 0)
    exact_ok = [p for p in ok if p["probe"] == "exact"]
    peak, peak_src = measured_peaks()
    line = {
        "metric": "QPS at recall@10=0.9 on 1 B300, low-prec batched vs FP32 plain; % HBM roofline",
        "value": best["qps"], "unit": "queries/s", "n_gpus": 1, "steps": max(3, min(args.steps, 5)),
        "warmup": 3, "ms_per_step": best["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16-lut/bf16-tc-gemm/f32-acc", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "nq": nq, "d": 128, "nlist": w.nlist, "M": w.M,
                   "k": k, "nprobe": best["nprobe"], "rerank_n": best["rerank_n"],
                   "probe": best["probe"] if best["probe"] == "exact" else
                   "navigation graph R %d S %d, entry %d, beam %d, max_check %d"
                   % (graph_info["R"], graph_info["S"], best["entry"], best["beam"], best["max_check"]),
                   "rerank": "Algorithm 1, BatchSize 32, eps -1, beta 1",
                   "raw_vectors": "HBM" if args.raw == "device" else "pinned host",
                   "replication": "Eq. 2, at most 8 lists, mean %.3f lists per vector"
                   % ((info.n + info.n_rep_entries) / info.n),
                   "clustering": "two-level k-means (%d iterations)" % min(args.kmeans_iters, 8)},
        "recall_at_10": best["recall_at_10"], "reaches_0_9": bool(ok),
        "best_exact_probe_qps": max(p["qps"] for p in exact_ok) if exact_ok else None,
        "graph": graph_info,
        "points": points,
        "replica_entries": int(info.n_rep_entries),
        "lists_per_vector": (info.n + info.n_rep_entries) / info.n,
        "duplicates_removed_per_query": best["gathered_per_query"] - best["distinct_per_query"],
        "index_device_bytes": int(info.device_bytes), "index_pinned_bytes": int(info.pinned_bytes),
        "build_s": t_build, "gen_s": t_gen, "gt_s": t_gt, "peak_hbm_gbs": peak, "peak_source": peak_src,
    }
    print(json.dumps(line))


def bench_spacev(args):
    """The SPACEV-like shape (Table 1): int8 d=100 vectors, M = 20, 25 or 50
    subspaces (scanned as 32 or 64 with zero padding subspaces), 16384 lists,
    10k queries, searched by the negated inner product (--metric ip) or
    squared L2. The precision form (FP16 table; tensor-core probe and LUT
    where d / M divides 16, FP32 SIMT otherwise) with an exhaustive re-rank of
    the ADC top-n on raw int8 rows in HBM, timed at each of --billion-points;
    the line reports the fastest point whose recall@10 (against brute force
    by the same metric) reaches 0.9."""
    import torch
    import oracle
    import paper_2409_16576_b300 as fa
    torch.cuda.set_device(0)
    w = synth.spacev_like(args.spacev_n, args.spacev_M)
    ip = args.metric == "ip"
    nq, k = w.nq, 10
    t0 = time.perf_counter()
    base = w.mix.base(w.n)
    queries = w.mix.queries(nq)
    t_gen = time.perf_counter() - t0
    bp = fa.build_params(nlist=w.nlist, M=w.M, kmeans_iters=min(args.kmeans_iters, 10),
                         raw_location=fa.FA_RAW_DEVICE, metric=fa.FA_METRIC_IP if ip else fa.FA_METRIC_L2)
    t0 = time.perf_counter()
    ix = fa.fa_build_index(base, bp)
    t_build = time.perf_counter() - t0
    ns = min(args.recall or 1000, nq)
    gt = ground_truth_u8(base, queries[:ns], 10, ip=ip)
    tc = 16 % (100 // w.M) == 0
    qd = torch.as_tensor(queries, device="cuda")
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    points = []
    for pt in args.billion_points.split(","):
        npb, n = (int(x) for x in pt.split(":"))
        g = fa.FA_GEMM_BF16_TC if tc else fa.FA_GEMM_SIMT_F32
        sp = fa.search_params(lut_prec=fa.FA_LUT_F16, lut_gemm=g, probe_gemm=g, rerank_n=n,
                              rerank_batch=32, rerank_eps=-1.0, rerank_beta=1)
        ms, tr = timed_steps(fa, torch, ix, qd, k, npb, sp, max(3, min(args.steps, 5)), 3, flush, oid, odist)
        found = oid.cpu().numpy()
        rec = oracle.recall_at(found[:ns], gt[0], gt[1], at=10)
        points.append({"nprobe": npb, "rerank_n": n, "qps": nq / (statistics.mean(ms) / 1e3),
                       "ms_per_step": statistics.mean(ms), "recall_at_10": rec,
                       "stage_ms": {"coarse": statistics.mean(t.coarse_ms for t in tr),
                                    "lut": statistics.mean(t.lut_ms for t in tr),
                                    "scan": statistics.mean(t.scan_ms for t in tr),
                                    "post": statistics.mean(t.post_ms for t in tr)}})
        print(json.dumps(points[-1]), flush=True)
    ok = [p for p in points if p["recall_at_10"] >= 0.9]
    best = max(ok, key=lambda p: p["qps"]) if ok else max(points, key=lambda p: p["recall_at_10"])
    print(json.dumps({
        "metric": "QPS at recall@10=0.9 on 1 B300, low-prec batched vs FP32 plain; % HBM roofline",
        "value": best["qps"], "unit": "queries/s", "n_gpus": 1, "steps": max(3, min(args.steps, 5)),
        "warmup": 3, "ms_per_step": best["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16-lut/%s/f32-acc" % ("bf16-tc-gemm" if tc else "f32-simt"),
        "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "nq": nq, "d": 100, "nlist": w.nlist, "M": w.M,
                   "scan_width": 32 if w.M <= 32 else 64, "metric": "inner product" if ip else "squared L2",
                   "k": k, "nprobe": best["nprobe"], "rerank_n": best["rerank_n"],
                   "rerank": "Algorithm 1, BatchSize 32, eps -1, beta 1", "raw_vectors": "HBM (int8)"},
        "recall_at_10": best["recall_at_10"], "reaches_0_9": bool(ok), "points": points,
        "build_s": t_build, "gen_s": t_gen}))


def exact_dists(base, q, ids):
    out = np.full(ids.shape, np.inf)
    for i in range(ids.shape[0]):
        ok = ids[i] >= 0
        x = base[ids[i][ok]].astype(np.float64)
        out[i, ok] = ((x - q[i].astype(np.float64)) ** 2).sum(1)
    return out


def err_vs_fp64(fa, oracle, ix, parts, base, queries, nprobe, sp, found_ids, found_dist, ns=16, npq=None):
    """Error of the GPU's distances against the FP64 oracle on the first ns
    queries: the form's ADC distances (its table precision, re-rank off, top
    100) against the oracle's ADC of the same ids (Eq. 1 in FP64), and the
    re-ranked distances of the bench's own results against the oracle's exact
    squared L2 of the same ids. Both as the largest relative error."""
    import ctypes
    p = fa.fa_search_params.from_buffer_copy(sp)
    p.rerank_n = 0
    p.flags &= ~fa.FA_GRAPH
    q = np.ascontiguousarray(queries[:ns])
    gi, gd = fa.fa_search_ex(ix, q, 100, nprobe, p, nprobe_per_query=npq)
    adc = 0.0
    for i in range(ns):
        ok = gi[i] >= 0
        ref = oracle.adc(oracle.lut(q[i], parts["codebooks"]), parts["codes"],
                         gi[i][ok].astype(np.uint32))
        adc = max(adc, float(np.max(np.abs(gd[i][ok] - ref) / np.maximum(ref, 1e-30))))
    out = {"adc_max_rel": adc, "sample": "first %d queries, ADC top-100 of the form's table" % ns}
    if sp.rerank_n > 0 and base is not None:
        rr = 0.0
        for i in range(ns):
            ok = found_ids[i] >= 0
            ref = oracle.exact_l2(q[i], base, found_ids[i][ok].astype(np.int64))
            rr = max(rr, float(np.max(np.abs(found_dist[i][ok] - ref) / np.maximum(ref, 1e-30))))
        out["rerank_max_rel"] = rr
        out["rerank"] = "exact (equal to FP64)" if rr == 0.0 else "FP32"
    return out


def search_params(fa, form, wl, persistent=False, serial=False):
    """plain: FP32 everywhere (SIMT coarse probe, FP32 LUT built in the scan CTA).
    lowp: BF16 tensor-core coarse probe and LUT GEMMs, FP16 (or FP8) LUT.
    Both forms re-rank the same top-n on exact FP32 distances (Algorithm 1)."""
    lowp = form in ("lowp", "batched")
    tc = fa.FA_GEMM_BF16_TC if lowp else fa.FA_GEMM_SIMT_F32
    prec = (fa.FA_LUT_FP8 if wl.get("lut") == "fp8" and form == "lowp" else fa.FA_LUT_F16) \
        if lowp else fa.FA_LUT_F32
    return fa.search_params(lut_prec=prec, lut_gemm=tc, probe_gemm=tc,
                            rerank_n=wl["rerank_n"], rerank_batch=wl["batch"],
                            rerank_beta=wl["beta"], rerank_eps=wl["eps"],
                            flags=(fa.FA_PERSISTENT if persistent else 0) | (fa.FA_SERIAL if serial else 0)
                            | (fa.FA_BATCHED if form == "batched" else 0))


def timed_steps(fa, torch, ix, qd, k, nprobe, sp, steps, warmup, flush, oid, odist):
    """Per-step CUDA events on the launching stream, L2 flushed between steps
    outside the events; returns (step ms list, traces)."""
    stream = torch.cuda.current_stream()

    def step(trace=None):
        fa.fa_search_ex(ix, qd, k, nprobe, sp, out_ids=oid, out_dist=odist,
                        stream=stream.cuda_stream, trace=trace)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    traces = []
    torch.cuda.nvtx.range_push("timed")  # lets ncu --nvtx-include "timed/" keep only these launches
    for i in range(steps):
        flush.zero_()
        tr = fa.fa_search_trace()
        ev[i][0].record(stream)
        step(tr)
        ev[i][1].record(stream)
        traces.append(tr)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return [x.elapsed_time(y) for x, y in ev], traces


def recall_of(oracle, base, queries, found, gt):
    ns = gt[0].shape[0]
    ex = exact_dists(base, queries[:ns], found[:ns])
    return oracle.recall_at(found[:ns], gt[0], gt[1], exact_found_dist=ex, at=10)


def main():
    args = parse()
    rank, world, local = dist_env()
    wl = workload(args)

    if args.impl == "reference":
        return reference_arm(args, wl, rank, world)
    if args.serve:
        return bench_serve(args)
    if args.workload == "zipf":
        return bench_zipf(args)
    if args.workload == "billion":
        return bench_billion(args)
    if args.workload == "spacev":
        return bench_spacev(args)

    import torch
    import oracle
    import paper_2409_16576_b300 as fa
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # ---- index (synthetic, seeded; the same on every replica) ----
    t0 = time.perf_counter()
    base = wl["mix"].base(wl["n"])
    q0, qn = replica_queries(rank, wl["nq"])
    queries = wl["mix"].queries(qn, start=q0)
    t_gen = time.perf_counter() - t0
    raw_loc = fa.FA_RAW_DEVICE if args.raw == "device" else fa.FA_RAW_HOST_PINNED
    bp = fa.build_params(nlist=wl["nlist"], M=wl["M"], kmeans_iters=args.kmeans_iters,
                         raw_location=raw_loc)
    t0 = time.perf_counter()
    ix = fa.fa_build_index(base, bp)
    t_build = time.perf_counter() - t0
    info = ix.info()

    k, nq, d = wl["k"], wl["nq"], 128
    qd = torch.as_tensor(queries, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    gt = ground_truth(base, queries[:min(args.recall, nq)], 10) if args.recall > 0 else None

    if args.sweep:
        return sweep(args, wl, fa, torch, oracle, ix, base, queries, qd, flush, gt, t_build)

    lowp = args.form in ("lowp", "batched")
    sp = search_params(fa, args.form, wl, args.persistent, args.serial)
    # the search pipelines scan and re-rank in 8 chunks when it re-ranks a large
    # batch from host memory (see FA_SERIAL in include/fa.h)
    pipelined = (wl["rerank_n"] > 0 and args.raw != "device" and not args.serial and not args.persistent
                 and wl["nq"] >= 4096)
    # autotuner: scan launch shape timed on a 2k-query sample of the batch
    tuned = fa.fa_autotune(ix, queries[:2000], k, wl["nprobe"], sp)["chosen"]
    pipelined = pipelined and tuned["tile_chunks"] == 0
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")

    # candidate counts (algorithmic bytes of the scan)
    _, _, st = fa.fa_search_ex(ix, queries, k, wl["nprobe"], sp, stats=True)
    uniq = int(st[:, 1].sum())
    gathered = int(st[:, 0].sum())
    rep_entries = gathered - uniq  # primaries are all distinct; the rest are replica entries
    ntop = max(wl["rerank_n"], k)
    lut_b = wl["M"] * 256 * (2 if lowp else 0)
    reranked = int(st[:, 3].sum())
    # an exhaustive re-rank of uint8 rows in HBM runs inside the selecting scan:
    # the stage then reads the re-ranked rows and writes no top-n rows
    fused = (wl["rerank_n"] > 256 and wl["eps"] < 0 and args.raw == "device" and k <= 32
             and not pipelined)
    scan_bytes = uniq * wl["M"] + rep_entries * 9 + nq * lut_b + (
        reranked * d if fused else nq * ntop * 8)

    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, traces = timed_steps(fa, torch, ix, qd, k, wl["nprobe"], sp, args.steps, args.warmup,
                                  flush, oid, odist)
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(step_ms), world, "cuda")
    value = world * nq / (ms / 1e3)
    scan_ms = statistics.mean(t.scan_ms for t in traces)
    launches = int(traces[0].launches) * args.steps

    # ---- e2e: host buffers through the C ABI, copies inside the region ----
    qh = torch.as_tensor(queries).pin_memory()
    ih = torch.empty((nq, k), dtype=torch.int64).pin_memory()
    dh = torch.empty((nq, k), dtype=torch.float32).pin_memory()
    qn, in_, dn = qh.numpy(), ih.numpy(), dh.numpy()
    for _ in range(2):
        fa.fa_search_ex(ix, qn, k, wl["nprobe"], sp, out_ids=in_, out_dist=dn)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fa.fa_search_ex(ix, qn, k, wl["nprobe"], sp, out_ids=in_, out_dist=dn)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_value = world * nq / (max_over_ranks(statistics.mean(e2e_ms), world, "cuda") / 1e3)

    recall = recall_of(oracle, base, queries, oid.cpu().numpy(), gt) if gt is not None else None
    parts = ix.parts()
    err = err_vs_fp64(fa, oracle, ix, parts, base, queries, wl["nprobe"], sp, oid[:16].cpu().numpy(),
                      odist[:16].cpu().numpy()) if rank == 0 else None

    # ---- roofline of the scan (dominant kernel) ----
    peak, peak_src = measured_peaks()
    achieved = scan_bytes / (scan_ms / 1e3) / 1e9
    khash = src_hash(SCAN_SOURCES)
    traffic = profile_traffic(khash, "%s-nq%d-nprobe%d-n%d" % (wl["name"], nq, wl["nprobe"], ntop))
    if ntop <= 256:
        scan_kernel = "k_scan"
    elif wl["rerank_n"] > 0 and wl["eps"] >= 0:
        scan_kernel = "k_scan_cta"  # an early-stopping re-rank reads sorted rows
    elif fused:
        scan_kernel = ("k_scan_sel with the exhaustive re-rank fused (+ k_scan_cta and k_rerank "
                       "for the queries it hands back)")
    else:
        scan_kernel = "k_scan_sel + k_scan_cta (the queries it hands back)"

    # ---- the plain FP32 form at the same operating point (same index) ----
    plain = None
    if lowp and not args.no_plain:
        spp = search_params(fa, "plain", wl, args.persistent, args.serial)
        fa.fa_autotune(ix, queries[:2000], k, wl["nprobe"], spp)
        pms, ptr = timed_steps(fa, torch, ix, qd, k, wl["nprobe"], spp, args.steps, args.warmup,
                               flush, oid, odist)
        pms = max_over_ranks(statistics.mean(pms), world, "cuda")
        precall = recall_of(oracle, base, queries, oid.cpu().numpy(), gt) if gt is not None else None
        plain = {"value": world * nq / (pms / 1e3), "ms_per_step": pms, "recall_at_10": precall,
                 "stage_ms": {"coarse": statistics.mean(t.coarse_ms for t in ptr),
                              "lut": statistics.mean(t.lut_ms for t in ptr),
                              "scan": statistics.mean(t.scan_ms for t in ptr),
                              "post": statistics.mean(t.post_ms for t in ptr)},
                 "what": "FP32 SIMT coarse probe, FP32 LUT built in the scan CTA, same re-rank"}

    # ---- the re-rank from the slow tier (the SSD stand-in) ----
    tiers = None
    if rank == 0 and world == 1 and lowp and wl["rerank_n"] > 0 and args.raw == "device" and not args.no_tiers:
        tiers = raw_tiers(fa, torch, oracle, parts, base, queries, gt, wl, sp, flush, args)

    # ---- CPU baseline: the oracle as it stands on a bounded sample ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ns = args.cpu_sample or 100
        secs, cores, _ = run_oracle_sample(wl, base, queries, parts, ns)
        cpu = {"value": ns / secs, "unit": "queries/s", "cores": cores, "kind": "oracle",
               "sample": "first %d of the %d queries, same index and parameters, FP64" % (ns, nq)}

    # ---- the batching form at its recall-0.9 point (its own index) ----
    batching = None
    if rank == 0 and world == 1 and not args.no_batching and args.workload == "sift10m":
        import copy
        za = copy.copy(args)
        # the batching workload at its configured size; an exhaustive re-rank of
        # the ADC top-256 on raw rows in HBM reaches recall@10 above 0.9 there
        za.zipf_n, za.zipf_rerank, za.steps, za.nq = args.batching_n, 256, min(args.steps, 5), 10_000
        za.with_serving = not args.no_serve
        za.recall = 1000
        zl = bench_zipf(za, emit=False)
        batching = {"workload": zl["config"]["workload"], "value": zl["value"], "unit": "queries/s",
                    "ms_per_step": zl["ms_per_step"], "recall_at_10": zl["recall_at_10"],
                    "plain_fp32": zl["plain_fp32_qps"], "recall_at_10_plain": zl["recall_at_10_plain"],
                    "lowp_over_plain": zl["speedup_vs_plain"],
                    "form": zl["config"]["form"] + "; BF16 tensor-core probe and LUT; exhaustive "
                            "re-rank of the ADC top-256 on raw rows in HBM",
                    "nprobe": "uniform 16..128 per query", "stage_ms": zl["stage_ms"],
                    "candidates_per_query": zl["candidates_per_query"],
                    "roofline": zl["roofline"], "err_vs_fp64": zl["err_vs_fp64"],
                    "serving_form": zl["serving_form"], "build_s": zl["build_s"]}

    if rank == 0:
        line = {
            "metric": "QPS at recall@10=0.9 on 1 B300, low-prec batched vs FP32 plain; % HBM roofline",
            "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("%s-lut/bf16-tc-gemm/f32-acc" % args.lut) if lowp else "f32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "n": wl["n"], "nq": nq, "d": d, "nlist": wl["nlist"],
                       "M": wl["M"], "nprobe": wl["nprobe"], "k": k, "form": args.form,
                       "rerank_n": wl["rerank_n"],
                       "rerank": "Algorithm 1, BatchSize %d, eps %g, beta %d" % (
                           wl["batch"], wl["eps"], wl["beta"]) if wl["rerank_n"] else "none",
                       "raw_vectors": ("HBM" if args.raw == "device" else "pinned host")
                       if wl["rerank_n"] else "none",
                       "parallelism": "replicas" if world > 1 else "single"},
            "l2": "flushed between timed steps (256 MB write); codes 320 MB > L2",
            "launch": "autotuned: %d threads/CTA, %d chunk(s) in flight per warp, %s" % (
                tuned["threads"], tuned["ilp"],
                "persistent" if (tuned["persistent"] or args.persistent) else "one CTA per query"),
            "recall_at_10": recall,
            "err_vs_fp64": err,
            "candidates_per_query": uniq / nq,
            "reranked_per_query": reranked / nq,
            "stage_ms": {"coarse": statistics.mean(t.coarse_ms for t in traces),
                         "lut": statistics.mean(t.lut_ms for t in traces), "scan": scan_ms,
                         "post": statistics.mean(t.post_ms for t in traces)},
            "plain_fp32": plain,
            "lowp_over_plain": (value / plain["value"]) if plain else None,
            "batching_form": batching,
            "raw_tiers": tiers,
            "roofline": {"bound": "hbm", "kernel": scan_kernel, "achieved": achieved, "peak": peak,
                         "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak,
                         "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic": traffic, "algorithmic_bytes_per_launch": scan_bytes,
                         "launches_per_step": 8 if pipelined else (2 if "k_scan_sel" in scan_kernel else 1),
                         "timed_as": ("the step's scan stage: 8 chunk launches on two streams, "
                                      "with the re-ranks of earlier chunks running beside them; "
                                      "bytes and traffic are the step's totals") if pipelined
                         else ("the step's scan stage: k_scan_sel (with the re-rank when fused) and "
                               "the k_scan_cta launch over the queries it hands back; bytes and "
                               "traffic are the stage's totals (candidate codes, LUT, and either "
                               "the re-ranked raw rows or the top-n rows)")
                         if "k_scan_sel" in scan_kernel else "the step's single scan launch",
                         "kernel_src_hash": khash},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": nq * d * 4,
                    "d2h_bytes_per_step": nq * k * 12},
            "gpu_launches": launches,
            "clocks": clk,
            "build_s": t_build, "gen_s": t_gen, "index_device_bytes": info.device_bytes,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def raw_tiers(fa, torch, oracle, parts, base, queries, gt, wl, sp, flush, args):
    """The same search with the raw vectors in the slow tier instead of HBM:
    rows in pinned host memory read over the host link in exact row pieces
    (the batch's re-ranks pipelined with its scans), and rows in §4.3's 4 KB
    pages (whole pages read, each page once per query: the paged re-rank) on
    a 1k-query sample, also at the configured point (top-100, eps 0, beta 2)."""
    k, nq, d = wl["k"], wl["nq"], 128
    out = {}
    pr = parts
    ixh = fa.fa_index_from_parts(pr["centroids"], pr["codebooks"], pr["codes"], pr["primary"], pr["rep_off"],
                                 pr["rep_ids"], raw=pr["raw"], raw_location=fa.FA_RAW_HOST_PINNED)
    qd = torch.as_tensor(queries, device="cuda")
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    ms, tr = timed_steps(fa, torch, ixh, qd, k, wl["nprobe"], sp, 3, 3, flush, oid, odist)
    _, _, st = fa.fa_search_ex(ixh, queries[:1000], k, wl["nprobe"], sp, stats=True)
    rows = float(st[:, 3].mean())
    t = statistics.mean(ms) / 1e3
    out["pinned_rows"] = {"qps": nq / t, "ms_per_step": t * 1e3,
                          "recall_at_10": recall_of(oracle, base, queries, oid.cpu().numpy(), gt),
                          "rows_per_query": rows, "link_gbs": nq * rows * d / t / 1e9,
                          "what": "raw rows in pinned host memory, read in 16-byte pieces over the host link; "
                                  "re-ranks of 8 query chunks pipelined with their scans"}
    del ixh
    ixp = fa.fa_index_from_parts(pr["centroids"], pr["codebooks"], pr["codes"], pr["primary"], pr["rep_off"],
                                 pr["rep_ids"], raw=pr["raw"], raw_location=fa.FA_RAW_HOST_PAGED)
    pm = fa.fa_debug_page_map(ixp)
    page_bytes = pm["rows_per_page"] * d
    ns = 1000
    for name, npb, spp in (("paged", wl["nprobe"], sp),
                           ("paged_configured_point", 64,
                            search_params(fa, "lowp", dict(rerank_n=100, batch=32, eps=0.0, beta=2)))):
        qs = torch.as_tensor(queries[:ns], device="cuda")
        o1 = torch.empty((ns, k), dtype=torch.int64, device="cuda")
        o2 = torch.empty((ns, k), dtype=torch.float32, device="cuda")
        ms, _ = timed_steps(fa, torch, ixp, qs, k, npb, spp, 2, 3, flush, o1, o2)
        reads = np.zeros(ns, np.int32)
        _, _, st = fa.fa_search_ex(ixp, queries[:ns], k, npb, spp, stats=True, page_reads=reads)
        t = statistics.mean(ms) / 1e3
        rec = recall_of(oracle, base, queries[:ns], o1.cpu().numpy(), gt) if gt is not None else None
        out[name] = {"qps": ns / t, "ms_per_step": t * 1e3, "queries_per_step": ns, "nprobe": npb,
                     "rerank_n": spp.rerank_n, "recall_at_10": rec,
                     "rows_reranked_per_query": float(st[:, 3].mean()) if spp.rerank_eps < 0 else None,
                     "minibatches_per_query": float(st[:, 2].mean()),
                     "pages_read_per_query": float(reads.mean()), "page_bytes": page_bytes,
                     "link_gbs": ns * float(reads.mean()) * page_bytes / t / 1e9,
                     "what": "raw rows in 4 KB pages (per-list buckets, max-min tail packing, §4.3); "
                             "whole pages read, each page once per query (intra- and inter-mini-batch "
                             "deduplication)"}
    del ixp
    return out


def zipf_form_name(args):
    return getattr(args, "zipf_form", "batched")


def zipf_form_desc(args):
    if zipf_form_name(args) == "batched":
        return ("batched list-major scan (FA_BATCHED: FP8 table, four queries per table word), "
                "CUDA graph")
    return "tiled persistent per-query scan (FP8 table expanded to FP32), CUDA graph, autotuned tiles"


def zipf_search_params(fa, args, rr, batch, extra=0):
    """The batching workload's forms: batch=True is the low-precision batched
    form (BF16 tensor-core probe and LUT, FP8 table; list-major or tiled
    scan), batch=False the plain FP32 form; both re-rank the ADC top-rr
    exhaustively when rr > 0."""
    tc = fa.FA_GEMM_BF16_TC
    r = dict(rerank_n=rr, rerank_eps=-1.0) if rr else {}
    if batch and zipf_form_name(args) == "batched":
        return fa.search_params(lut_prec=fa.FA_LUT_FP8, lut_gemm=tc, probe_gemm=tc,
                                flags=extra | fa.FA_BATCHED, **r)
    if batch:
        return fa.search_params(lut_prec=fa.FA_LUT_FP8, lut_gemm=tc, probe_gemm=tc,
                                flags=extra | fa.FA_PERSISTENT, **r)
    return fa.search_params(flags=extra, **r)


def bench_zipf(args, emit=True):
    """Batching form on uneven work: unit-norm d=96 vectors in 65536 lists of
    Zipf(1.1) sizes (the largest holds ~14% of the base), 10k queries with
    nprobe uniform in 16..128, k 10, M 48. The batching form (BF16 tensor-core
    probe and LUT, FP8 LUT, tiled persistent scan, CUDA graph, autotuned tile
    size) against the plain FP32 form (one CTA per query) on the same index."""
    import ctypes
    import torch
    import oracle
    import paper_2409_16576_b300 as fa
    torch.cuda.set_device(0)
    z = synth.ZipfLists(args.zipf_n)
    nq, k, M = args.nq, 10, 48
    t0 = time.perf_counter()
    base = z.base()
    cent, prim = z.centroids(), z.primary()
    queries = z.queries(nq)
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    rr = args.zipf_rerank
    ix = fa.fa_build_index_lists(base, cent, prim, fa.build_params(
        M=M, kmeans_iters=args.kmeans_iters, raw_location=fa.FA_RAW_DEVICE if rr else fa.FA_RAW_NONE))
    t_build = time.perf_counter() - t0
    npq = synth.uniform_ints(16, 128, nq, tag=3)
    npq_d = torch.as_tensor(npq, device="cuda")
    qd = torch.as_tensor(queries, device="cuda")
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    tc = fa.FA_GEMM_BF16_TC

    def params(batch, extra=0):
        return zipf_search_params(fa, args, rr, batch, extra)

    # autotune the batching form (tile size, threads) on host copies of a sample
    sp_t = params(True)
    npq_h = np.ascontiguousarray(npq[:2000])
    sp_t.nprobe_per_query = npq_h.ctypes.data_as(ctypes.c_void_p)
    tuned = fa.fa_autotune(ix, queries[:2000], k, 128, sp_t)["chosen"]
    _, _, st = fa.fa_search_ex(ix, queries, k, 128, params(True), nprobe_per_query=npq, stats=True)
    cand = st[:, 1].astype(np.int64)

    def timed(sp, steps):
        stream = torch.cuda.current_stream()
        run = lambda: fa.fa_search_ex(ix, qd, k, 128, sp, out_ids=oid, out_dist=odist,
                                      nprobe_per_query=npq_d, stream=stream.cuda_stream)
        for _ in range(3):
            run()
        torch.cuda.synchronize()
        ms = []
        torch.cuda.nvtx.range_push("timed")
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        torch.cuda.nvtx.range_pop()
        return statistics.mean(ms)

    clocks = ClockSampler(0)
    clocks.start()
    ms_batch = timed(params(True, fa.FA_GRAPH), args.steps)
    clk = clocks.stop()
    ids_batch = oid.cpu().numpy()
    dist_batch = odist.cpu().numpy()
    ms_plain = timed(params(False), max(3, args.steps // 4))
    ids_plain = oid.cpu().numpy()
    tr = fa.fa_search_trace()
    fa.fa_search_ex(ix, qd, k, 128, params(True), out_ids=oid, out_dist=odist,
                    nprobe_per_query=npq_d, trace=tr)
    ns = min(args.recall, nq) if args.recall else 0
    rec_b = rec_p = None
    gt = None
    if ns:
        gt = ground_truth(base, queries[:ns], 10)
        rec_b = recall_of(oracle, base, queries, ids_batch, gt)
        rec_p = recall_of(oracle, base, queries, ids_plain, gt)
    peak, peak_src = measured_peaks()
    scan_bytes = int(cand.sum()) * M + nq * M * 256 + nq * 10 * 8
    batched = zipf_form_name(args) == "batched"
    # the scan's bound is its shared-memory table reads, not HBM: one 32-bit
    # table word per (candidate, subspace) serves G queries (4 FP8 entries in
    # the batched form, 1 FP32 entry in the tiled per-query scan); the peak is
    # one 128-byte shared-memory wavefront per clock per SM
    G = 4 if batched else 1
    table_bytes = int(cand.sum()) * M * 4 // G
    props = torch.cuda.get_device_properties(0)
    sm_mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2032.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2032.0
    smem_peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e9
    wl_key = "ivfpq-f32unit-%dm-d96-zipf65536-M48-nq%d-rr%d-%s" % (args.zipf_n // 1_000_000, nq, rr,
                                                                     zipf_form_name(args))
    dram = profile_traffic(src_hash(SCAN_SOURCES), wl_key)
    err = None
    if getattr(args, "zipf_err", True):
        parts = ix.parts(with_raw=False)
        err = err_vs_fp64(fa, oracle, ix, parts, base if rr else None, queries, 128, params(True),
                          ids_batch[:16], dist_batch[:16], npq=npq[:16])
        del parts
    serving = None
    if getattr(args, "with_serving", False):
        pool = z.queries(20000)
        srv, sres, sstats = serve_load(fa, ix, params(True), pool,
                                       [float(r) for r in args.rates.split(",")],
                                       args.serve_seconds, args.window_us)
        srec = serve_recall(srv, pool, gt) if ns else None
        srv.close()
        serving = {"loads": sres, **sstats, "recall_at_10": srec, "k": "uniform {1,10,100}",
                   "nprobe": "uniform 32..256", "window_us": args.window_us, "max_batch": 4096,
                   "rerank_n": rr, "recall_requests": "k 10, nprobe uniform 32..256, %d queries" % ns}
    line = {
        "metric": "QPS at recall@10=0.9 on 1 B300, low-prec batched vs FP32 plain; % HBM roofline",
        "value": nq / (ms_batch / 1e3), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": 3, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp8-lut/bf16-tc-gemm/f16x2-then-f32-acc" if zipf_form_name(args) == "batched"
        else "fp8-lut/bf16-tc-gemm/f32-acc", "data": "synthetic",
        "config": {"workload": "ivfpq-f32unit-%dm-d96-zipf65536-M48" % (args.zipf_n // 1_000_000),
                   "n": args.zipf_n, "nq": nq, "nlist": 65536, "M": M, "k": k,
                   "nprobe": "uniform 16..128 per query", "form": zipf_form_desc(args),
                   "rerank_n": rr, "rerank": "Algorithm 1 exhaustive (eps < 0), raw rows in HBM" if rr else "none",
                   "tuned": tuned, "l2": "flushed between timed steps"},
        "plain_fp32_qps": nq / (ms_plain / 1e3), "speedup_vs_plain": ms_plain / ms_batch,
        "recall_at_10": rec_b, "recall_at_10_plain": rec_p,
        "candidates_per_query": {"mean": float(cand.mean()), "max": int(cand.max()),
                                 "min": int(cand.min())},
        "largest_list_fraction": float(z.sizes().max() / args.zipf_n),
        "stage_ms": {"coarse": tr.coarse_ms, "lut": tr.lut_ms, "scan": tr.scan_ms, "post": tr.post_ms},
        "roofline": {"bound": "alu",
                     "kernel": "k_bq_scan (+ k_bq_tau, k_bq_select)" if batched else "k_scan (tiled)",
                     "achieved": table_bytes / (tr.scan_ms / 1e3) / 1e9, "peak": smem_peak,
                     "peak_source": "derived: %d SMs x 128 B shared-memory wavefront per clock x %.0f MHz"
                     % (props.multi_processor_count, sm_mhz),
                     "unit": "GB/s", "frac": table_bytes / (tr.scan_ms / 1e3) / 1e9 / smem_peak,
                     "traffic": dram,
                     "what": "shared-memory table bytes the scan stage must read (one 32-bit word per "
                             "(candidate, subspace) for every %d queries) over the stage's time" % G,
                     "hbm": {"dram_gbs": (dram / (tr.scan_ms / 1e3) / 1e9) if dram else None,
                             "peak": peak, "peak_source": peak_src,
                             "frac": (dram / (tr.scan_ms / 1e3) / 1e9 / peak) if dram else None,
                             "per_query_code_bytes_gbs": scan_bytes / (tr.scan_ms / 1e3) / 1e9,
                             "note": "code bytes counted once per (query, candidate) exceed the DRAM "
                                     "traffic: a list is read once for a group of queries and from L2"},
                     "algorithmic_bytes_per_launch": table_bytes, "traffic_workload": wl_key},
        "err_vs_fp64": err, "serving_form": serving,
        "clocks": clk, "build_s": t_build, "gen_s": t_gen,
    }
    ix.free()
    if emit:
        print(json.dumps(line))
    return line


def serve_load(fa, ix, sp, pool, rates, seconds, window_us, max_batch=4096, slots=4):
    """Open-loop Poisson load on the request loop (fa_server_*) over ix: at
    each offered rate, requests with k uniform in {1, 10, 100} and nprobe
    uniform in 32..256 arrive with seeded exponential gaps; returns sustained
    QPS (completed / elapsed), p50, p99 and mean latency from submit to
    completion per rate, and the loop's statistics."""
    import threading as th
    srv = fa.Server(ix, sp, max_batch=max_batch, window_us=window_us, slots=slots, kmax=100,
                    nprobe_max=256)
    results = []
    for rate in rates:
        count = int(rate * seconds)
        arr = synth.poisson_arrivals(rate, count)
        ks = np.array([1, 10, 100], dtype=np.int32)[synth.uniform_ints(0, 2, count, tag=11)]
        nps = synth.uniform_ints(32, 256, count, tag=12)
        qi = np.arange(count) % pool.shape[0]
        lat = np.empty(count)
        done_t = [0.0]
        got = [0]

        def collect():
            while got[0] < count:
                rid, _, _, l, st = srv.poll(max_results=8192, timeout_us=2000)
                if rid.shape[0]:
                    lat[got[0]:got[0] + rid.shape[0]] = l
                    got[0] += rid.shape[0]
                    done_t[0] = time.perf_counter()

        c = th.Thread(target=collect)
        c.start()
        start = time.perf_counter()
        i = 0
        while i < count:
            now = time.perf_counter() - start
            j = int(np.searchsorted(arr, now, side="right"))
            if j > i:
                srv.submit(pool[qi[i:j]], ks[i:j], nps[i:j])
                i = j
            else:
                time.sleep(min(2e-4, max(0.0, arr[i] - now)))
        c.join()
        elapsed = done_t[0] - start
        results.append({"offered_qps": rate, "requests": count,
                        "sustained_qps": count / elapsed, "p50_ms": float(np.percentile(lat, 50)) / 1e3,
                        "p99_ms": float(np.percentile(lat, 99)) / 1e3,
                        "mean_ms": float(lat.mean()) / 1e3})
        if results[-1]["sustained_qps"] < 0.5 * rate:
            break  # far beyond capacity: higher rates only grow the queue
    st = srv.stats()
    stats = {"batches": st.batches, "requests": st.requests, "slots": st.slots,
             "slot_device_bytes": st.device_bytes}
    return srv, results, stats


def serve_recall(srv, queries, gt, k=10, nprobe=None):
    """recall@10 of requests served by srv (k 10, nprobe uniform in 32..256)
    on the ground-truth subsample."""
    import oracle
    ns = gt[0].shape[0]
    nps = synth.uniform_ints(32, 256, ns, tag=13) if nprobe is None else np.full(ns, nprobe, np.int32)
    rid = srv.submit(queries[:ns], np.full(ns, k, np.int32), nps)
    pos = {int(r): i for i, r in enumerate(rid)}
    found = np.full((ns, k), -1, np.int64)
    got = 0
    while got < ns:
        r, ids, _, _, st = srv.poll(max_results=8192, timeout_us=20000)
        for j in range(r.shape[0]):
            found[pos[int(r[j])]] = ids[j][:k]
        got += r.shape[0]
    return oracle.recall_at(found, gt[0], gt[1], at=10)


def bench_serve(args):
    """Serving form on the Zipf-lists index (standalone): see serve_load."""
    import paper_2409_16576_b300 as fa
    import torch
    torch.cuda.set_device(0)
    z = synth.ZipfLists(args.zipf_n)
    t0 = time.perf_counter()
    base = z.base()
    rr = args.zipf_rerank
    ix = fa.fa_build_index_lists(base, z.centroids(), z.primary(), fa.build_params(
        M=48, kmeans_iters=args.kmeans_iters, raw_location=fa.FA_RAW_DEVICE if rr else fa.FA_RAW_NONE))
    t_build = time.perf_counter() - t0
    pool = z.queries(20000)
    sp = zipf_search_params(fa, args, rr, batch=True)
    gt = ground_truth(base, pool[:min(args.recall, 1000)], 10) if args.recall else None
    del base
    srv, results, stats = serve_load(fa, ix, sp, pool, [float(r) for r in args.rates.split(",")],
                                     args.serve_seconds, args.window_us)
    rec = serve_recall(srv, pool, gt) if gt is not None else None
    srv.close()
    print(json.dumps({"serving": results, **stats, "recall_at_10": rec,
                      "config": {"workload": "ivfpq-f32unit-%dm-d96-zipf65536-M48" % (args.zipf_n // 1_000_000),
                                 "k": "uniform {1,10,100}", "nprobe": "uniform 32..256",
                                 "window_us": args.window_us, "max_batch": 4096, "slots": 4,
                                 "rerank_n": rr, "form": zipf_form_name(args)},
                      "build_s": t_build}))


def sweep(args, wl, fa, torch, oracle, ix, base, queries, qd, flush, gt, t_build):
    """QPS and recall@10 over a grid of operating points (one index build)."""
    k, nq = wl["k"], wl["nq"]
    oid = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    odist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    # IVF coverage: share of the true 10-NN inside the nprobe nearest lists
    if gt is not None:
        ns = gt[0].shape[0]
        primary = ix.parts()["primary"]
        probes = fa.fa_debug_probes(ix, queries[:ns], 512)
        for npb in (8, 16, 32, 64, 128, 256, 512):
            cov = np.mean([np.isin(primary[gt[0][i]], probes[i, :npb]).mean() for i in range(ns)])
            print(json.dumps({"coverage_nprobe": npb, "coverage": float(cov)}), flush=True)
    if args.points:
        grid = []
        for pt in args.points.split(","):
            f, npb, n, batch, eps, beta = pt.split(":")
            grid.append((f, int(npb), int(n), int(batch), float(eps), int(beta)))
    else:
        grid = [("lowp", 64, 100, 32, 0.0, 2), ("plain", 64, 100, 32, 0.0, 2)]  # the configured point
        for form in ("lowp", "plain"):
            for npb in (64, 128, 256, 512):
                for n in (1024, 4096, 16384):
                    grid.append((form, npb, n, 32, -1.0, 1))
        for npb in (128, 256):
            grid.append(("lowp", npb, 16384, 32, 0.0, 2))
    for form, npb, n, batch, eps, beta in grid:
        w = dict(wl, rerank_n=n, batch=batch, eps=eps, beta=beta)
        sp = search_params(fa, form, w)
        ms, tr = timed_steps(fa, torch, ix, qd, k, npb, sp, 3, 3, flush, oid, odist)
        r = recall_of(oracle, base, queries, oid.cpu().numpy(), gt) if gt is not None else None
        print(json.dumps({"form": form, "nprobe": npb, "rerank_n": n, "batch": batch, "eps": eps,
                          "beta": beta, "qps": nq / (statistics.mean(ms) / 1e3),
                          "ms": statistics.mean(ms), "recall_at_10": r,
                          "stage_ms": [statistics.mean(t.coarse_ms for t in tr),
                                       statistics.mean(t.lut_ms for t in tr),
                                       statistics.mean(t.scan_ms for t in tr),
                                       statistics.mean(t.post_ms for t in tr)]}), flush=True)


def reference_arm(args, wl, rank, world):
    """The FP64 CPU oracle as the reference implementation: each step is a
    bounded sample of the workload's queries against the same index."""
    if rank != 0:
        return
    import oracle
    import paper_2409_16576_b300 as fa  # only to build the index both arms search
    import torch
    torch.cuda.set_device(0)
    base = wl["mix"].base(wl["n"])
    queries = wl["mix"].queries(wl["nq"])
    bp = fa.build_params(nlist=wl["nlist"], M=wl["M"], kmeans_iters=args.kmeans_iters,
                         raw_location=fa.FA_RAW_HOST_PINNED)
    ix = fa.fa_build_index(base, bp)
    parts = ix.parts()
    ns = args.cpu_sample or 32
    times = []
    for i in range(max(3, args.warmup) + args.steps):
        secs, cores, _ = run_oracle_sample(wl, base, queries[(i * ns) % wl["nq"]:], parts, ns)
        if i >= max(3, args.warmup):
            times.append(secs)
    ms = statistics.mean(times) * 1e3
    v = ns / (ms / 1e3)
    print(json.dumps({
        "impl": "reference",
        "metric": "QPS at recall@10=0.9 on 1 B300, low-prec batched vs FP32 plain; % HBM roofline",
        "value": v, "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "n": wl["n"], "nq": wl["nq"], "d": 128,
                   "nlist": wl["nlist"], "M": wl["M"], "nprobe": wl["nprobe"], "k": wl["k"],
                   "form": args.form, "rerank_n": wl["rerank_n"],
                   "rerank": "Algorithm 1, BatchSize %d, eps %g, beta %d" % (
                       wl["batch"], wl["eps"], wl["beta"]) if wl["rerank_n"] else "none",
                   "raw_vectors": ("HBM" if args.raw == "device" else "pinned host")
                   if wl["rerank_n"] else "none",
                   "parallelism": "single"},
        "cpu_baseline": {"value": v, "unit": "queries/s", "kind": "oracle", "cores": cpu_cores(),
                         "sample": "%d queries per step" % ns},
        "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
