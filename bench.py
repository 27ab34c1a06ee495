"""Benchmark: LeaFi-enhanced DSTree k-NN search on one B300 (weak-scaled replicas for N > 1).

Workload (batched 1-NN search): N = 1,000,000 z-normalised random walks of
length 256 (float32, 1.02 GB resident, larger than L2), DSTree leaf capacity
10,000, MLP filters on the 100 largest leaves trained on 2,000 queries
(1,500 global + 500 local per leaf) and auto-tuned for 1-NN, then 10,000
noise-perturbed queries (10/20/30/40% noise) searched in launches of 256 at a
99% recall target.  One step = the whole query set (40 launches).  The plain
summarisation-bound search of the same index (exact mode) is timed beside it.

Prints one JSON line (rank 0).  `--impl reference` times the oracle (plain C
restatement, host cores) on bounded samples of the same workload instead.

`--config` selects other measurement configurations, each printing its own
JSON line (not the headline): `serving` (Poisson arrivals into the request
loop, per-query k and recall target, p50/p99 latency), `mixed` (iSAX over
uneven leaves, k in {1, 10, 100}, targets in {0.9, 0.95, 0.99}, with the
training-target generation timed as a build phase) and `precision`
(embedding-like m = 96, k = 10: tensor-core vs CUDA-core scan, error against
float64, and the flat contraction over all series as the tensor-core case).
"""
from __future__ import annotations

import argparse
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

import fixtures as fx  # noqa: E402

M = 256
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}
SMS = 148
FP32_LANES = 128
# DRAM bytes (read + write) per tensor-core leaf-scan launch on the default
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# every scan launch of the timed LeaFi region at W = 64, averaged), valid only
# for the kernel code it was taken on (SHA-1 of k_scan_tc.cu up to the round
# prep/finish kernels, i.e. the scan kernel and its device helpers, without
# comments and blank lines)
SCAN_TRAFFIC = {"bytes_per_launch": 161.0e6, "kernel_sha1": "e1d99332fdb972dfedf94e76f77cb45df8e42e50",
                "source": "stored ncu capture (profiles/leaf_scan_tc_dram_1M.md), not measured "
                          "in this run"}


def code_sha1(path, stop=None):
    """Hash of a source file without comments and blank lines; with `stop`, of
    the text before its first occurrence only (the leaf-scan kernel and its
    device helpers precede the round prep/finish kernels in their file)."""
    import hashlib
    import re
    with open(path, encoding="utf-8") as f:
        src = f.read()
    if stop is not None and stop in src:
        src = src[:src.index(stop)]
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
    return hashlib.sha1(src.encode()).hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="leafi", choices=["leafi", "reference"])
    ap.add_argument("--config", default="batched",
                    choices=["batched", "serving", "mixed", "precision", "ablation", "cnn"])
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--queries", type=int, default=10_000)
    ap.add_argument("--launch", type=int, default=256)
    ap.add_argument("--filters", type=int, default=None)
    ap.add_argument("--leaf-cap", type=int, default=None)
    ap.add_argument("--rates", default="1000,5000,10000,20000,50000",
                    help="serving: Poisson arrival rates, queries/s")
    ap.add_argument("--seconds", type=float, default=1.0, help="serving: arrivals per rate")
    ap.add_argument("--max-wait-ms", type=float, default=0.2)
    ap.add_argument("--scan-path", type=int, default=0, help="0 tensor-core scan, 1 CUDA-core scan")
    ap.add_argument("--epochs", type=int, default=1000)
    ap.add_argument("--wave", type=int, default=None,
                    help="leaves per wave (64; 512 for the iSAX configuration's small leaves)")
    ap.add_argument("--target", type=float, default=0.99)
    ap.add_argument("--cpu-sample", type=int, default=3072,
                    help="queries of the oracle's timed sample (about 12 s on 16 host threads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-schedule", action="store_true",
                    help="batches in the callers' query order (no route-leaf scheduling)")
    ap.add_argument("--lanes", type=int, default=8, help="batches of one call in flight")
    ap.add_argument("--batch", type=int, default=None,
                    help="queries per internal batch of a call (default: --launch)")
    ap.add_argument("--part", type=int, default=2048, help="series per leaf-scan work item")
    ap.add_argument("--items-per-sm", type=int, default=4,
                    help="scan work items per SM a round aims at (0: fixed part)")
    ap.add_argument("--min-part", type=int, default=512,
                    help="smallest series per work item a round may take")
    ap.add_argument("--scan-blocks", type=int, default=0,
                    help="thread blocks per tensor-core scan launch (0: one per SM)")
    a = ap.parse_args()
    dflt = {"batched": (1_000_000, 10_000, 100), "ablation": (1_000_000, 10_000, 100),
            "cnn": (1_000_000, 10_000, 100),
            "serving": (50_000_000, 10_000, 1000),
            "mixed": (25_000_000, 20_000, 1000), "precision": (10_000_000, 10_000, 0)}[a.config]
    a.n = a.n if a.n is not None else dflt[0]
    a.leaf_cap = a.leaf_cap if a.leaf_cap is not None else dflt[1]
    a.filters = a.filters if a.filters is not None else dflt[2]
    # waves: 64 leaves per query on the 1M random walks; the precision,
    # mixed-k and serving searches take every remaining leaf after the route
    # leaf in one wave (measured: narrow waves re-read the same leaves for few
    # queries each)
    # wave width: given, or chosen by the library's search-schedule autotuner
    # while the filters are built (the initial width below is only its start)
    a.tune = a.wave is None
    a.wave = a.wave if a.wave is not None else {"mixed": 65536, "precision": 4096,
                                                "serving": 16384}.get(a.config, 64)
    return a


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region (clocks and throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.nearest = False

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark(self, t0, t1):
        """Keep the samples that arrived in [t0, t1] (plus one sampling period);
        if none did, the nearest sample on either side."""
        inside = [x for x in self.lines if t0 <= x[0] <= t1 + 0.1]
        if not inside and self.lines:
            before = [x for x in self.lines if x[0] < t0][-1:]
            after = [x for x in self.lines if x[0] > t1][:1]
            inside = before + after
            self.nearest = True
        self.lines = inside

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if self.nearest:
            out["note"] = "timed region shorter than the sampling period: nearest samples"
        return out


def dist_setup(gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        # one process per GPU over NCCL; gloo where there is no GPU (host-side tests)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local, dist


def max_over_ranks(x, dist, device):
    if dist is None:
        return x
    import torch
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def workload_config(a):
    return {"workload": "batched 1-NN LeaFi-DSTree search, N=%d random walks, m=%d, "
                        "leaf capacity %d, %d filters, %d queries in launches of %d, recall target %.2f"
                        % (a.n, M, a.leaf_cap, a.filters, a.queries, a.launch, a.target),
            "n_series": a.n, "length": M, "leaf_capacity": a.leaf_cap, "filters": a.filters,
            "queries": a.queries, "launch": a.launch, "recall_target": a.target,
            "k": 1, "wave": a.wave if not getattr(a, "tune", False) else "autotuned",
            "schedule": "route-leaf order" if not getattr(a, "no_schedule", False) else "caller order",
            "lanes": getattr(a, "lanes", 8), "part": getattr(a, "part", 2048),
            "items_per_sm": getattr(a, "items_per_sm", 4),
            "min_part": getattr(a, "min_part", 512),
            "scan_blocks": getattr(a, "scan_blocks", 0),
            "scan_path": {0: "float16 tensor cores", 1: "CUDA cores",
                          2: "e4m3 tensor cores"}.get(getattr(a, "scan_path", 0)),
            "l2": "inputs larger than L2 (%.2f GB float32 series, %.2f GB float16 copy)"
                  % (a.n * M * 4 / 1e9, a.n * M * 2 / 1e9)}


def clock_mhz(clocks, fallback):
    return clocks.get("sm_mhz") or fallback


def cpu_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def oracle_leafi_rate(X, fl, W, alpha, qp, Q, leaf_cap, wave, target, sample):
    """Time the oracle's LeaFi search on `sample` queries (bounded CPU work)."""
    import oracle as O
    t = O.Tree(X, "dstree", leaf_cap=leaf_cap, init_segments=4)
    j = O.offset_position(qp, target)
    Qs = np.ascontiguousarray(Q[:sample])
    t0 = time.perf_counter()
    O.leafi_search(t, W, fl, alpha, Qs, 1, j, wave)
    dt = time.perf_counter() - t0
    return sample / dt, dt, t


def run_reference(a):
    """Oracle arm: the plain CPU restatement, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    oracle_build = O.build()
    X = fx.random_walk(a.n, M)
    Q = fx.test_queries(X, a.queries)
    t = O.Tree(X, "dstree", leaf_cap=a.leaf_cap, init_segments=4)
    # the oracle trains its own filters on the same draws (a short schedule keeps it bounded)
    sizes = t.leaf_sizes()
    F = min(a.filters, t.L)
    fl = np.array(sorted(range(t.L), key=lambda l: (-sizes[l], l))[:F], np.int32)
    # Alg. 1's draws from the oracle's own generator, with the library's default seed
    seed = 2502018361
    W = O.filter_init(F, M, M, seed)
    Qg, Ql, _, _ = O.training_queries(t, fl, 1500, 500, 0.1, 0.4, seed)
    Tg, Tl = O.train_targets(t, fl, Qg, Ql)
    p = O.TrainParams(max_epochs=3)
    Wt, _, _ = O.train(p, Qg, Tg, Ql, Tl, O.epoch_perms(3, 1600, seed), *W)
    alpha, qp = O.fit_autotuner(t, Wt, fl, Qg[1200:], 1, a.wave)
    j = O.offset_position(qp, a.target)
    per = max(4, min(a.cpu_sample, 64))  # per step: a whole run stays within a minute
    times = []
    for s in range(a.warmup + a.steps):
        Qs = np.ascontiguousarray(Q[(s * per) % a.queries:][:per])
        t0 = time.perf_counter()
        O.leafi_search(t, Wt, fl, alpha, Qs, 1, j, a.wave)
        if s >= a.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    value = per / (ms / 1e3)
    line = {"impl": "reference", "metric": "queries/s at 99% recall (LeaFi search)",
            "value": value, "unit": "queries/s", "n_gpus": 0, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(a),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cpu_threads(),
                             "kind": "oracle",
                             "sample": "%d queries per step of the same workload (oracle filters "
                                       "trained 3 epochs)" % per},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- other configurations
def _gpu_setup():
    import torch
    torch.cuda.set_device(0)
    import paper_2502_01836_b300 as lf
    return torch, lf


def _emit(line):
    print(json.dumps(line), flush=True)


def run_serving(a):
    """Poisson arrivals of single-query requests, k ~ U{1..100}, target in
    {0.9, 0.95, 0.99, exact}, into the request loop over a resident index."""
    torch, lf = _gpu_setup()
    from paper_2502_01836_b300.workflow import enhance
    t0 = time.perf_counter()
    X = fx.random_walk(a.n, M)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=a.leaf_cap, wave=a.wave, device=0))
    t_build = time.perf_counter() - t0
    info = lf.leafi_get_info(idx)
    F = min(a.filters, info.n_leaves)
    t0 = time.perf_counter()
    enhance(idx, F, kclasses=(1, 10, 100), max_epochs=a.epochs, tune_search=int(a.tune))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    kmax = 100
    lf.leafi_set_profiling(idx, 2)
    sv = lf.leafi_serve_start(idx, kmax=kmax, max_batch=a.batch or a.launch,
                              max_wait_ms=a.max_wait_ms)
    rows = []
    try:
        for ri, lam in enumerate(float(x) for x in a.rates.split(",")):
            n = int(min(40_000, max(200, lam * a.seconds)))
            rng = np.random.default_rng(2502 + ri)
            arrive = np.cumsum(rng.exponential(1.0 / lam, n))
            ks = rng.integers(1, kmax + 1, n).astype(np.int32)
            tg = rng.choice([0.9, 0.95, 0.99, 1.0], n).astype(np.float64)
            Q = fx.test_queries(X, n, seed=fx.SEED_TEST + 100 + ri)
            tickets = [None] * n
            ready = threading.Event()
            st0 = lf.leafi_serve_get_stats(sv)

            def submitter():
                base = time.perf_counter()
                ready.set()
                for i in range(n):
                    while time.perf_counter() - base < arrive[i]:
                        pass
                    while True:
                        try:
                            tickets[i] = lf.leafi_serve_submit(sv, Q[i:i + 1], ks[i:i + 1],
                                                               tg[i:i + 1])
                            break
                        except lf.LeafiError as e:
                            if e.status != lf.EAGAIN:
                                raise
                            time.sleep(1e-4)
                sub_done[0] = time.perf_counter() - base

            sub_done = [0.0]
            th = threading.Thread(target=submitter)
            th.start()
            ready.wait()
            t_start = time.perf_counter()
            ids = np.zeros((1, kmax), np.int64)
            dd = np.zeros((1, kmax), np.float32)
            lat = np.zeros(n)
            for i in range(n):
                while tickets[i] is None:
                    time.sleep(1e-5)
                while True:
                    done, l_ms = lf.leafi_serve_poll(sv, tickets[i], ids, dd, wait_ms=100.0)
                    if done:
                        lat[i] = l_ms
                        break
            elapsed = time.perf_counter() - t_start
            th.join()
            st1 = lf.leafi_serve_get_stats(sv)
            nb = st1["batches"] - st0["batches"]
            rows.append({"offered_qps": lam, "requests": n, "achieved_qps": n / elapsed,
                         "offered_span_s": float(arrive[-1]), "submit_span_s": sub_done[0],
                         "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)),
                         "batches": nb, "mean_batch": n / max(nb, 1)})
        sst = lf.leafi_serve_get_stats(sv)
    finally:
        lf.leafi_serve_stop(sv)
    kt = lf.leafi_get_kernel_times(idx)
    lf.leafi_set_profiling(idx, 0)
    _emit({"metric": "serving: latency and throughput under Poisson arrivals", "unit": "queries/s",
           "kernel_ms_total": {k: [v[0], v[1]] for k, v in kt.items() if v[1]},
           "server_stats": sst,
           "config": {"workload": "DSTree over %d random walks x %d, leaf capacity %d, filters on "
                                  "the %d largest leaves, single-query requests with k ~ U{1..100} "
                                  "and target in {0.9, 0.95, 0.99, exact}" % (a.n, M, a.leaf_cap, F),
                      "leaves": info.n_leaves, "max_batch": a.batch or a.launch,
                      "max_wait_ms": a.max_wait_ms,
                      "wave": lf.leafi_get_info(idx).wave, "tuned": bool(a.tune)},
           "rates": rows, "data": "synthetic",
           "build_s": {"data": t_data, "index": t_build, "train_and_tune": t_train},
           "device_bytes": info.device_bytes})
    lf.leafi_free(idx)


def run_mixed(a):
    """iSAX over uneven leaves; k in {1, 10, 100}, targets in {0.9, 0.95, 0.99};
    training-target generation (per-query per-leaf nearest distance) timed."""
    torch, lf = _gpu_setup()
    from paper_2502_01836_b300.workflow import enhance
    t0 = time.perf_counter()
    X = fx.random_walk(a.n, M)
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    idx = lf.leafi_build(X, lf.BuildParams(index_type=lf.ISAX, leaf_capacity=a.leaf_cap,
                                           wave=a.wave, device=0, scan_path=a.scan_path))
    t_build = time.perf_counter() - t0
    info = lf.leafi_get_info(idx)
    sizes = lf.leafi_leaf_sizes(idx)
    F = min(a.filters, info.n_leaves)
    fl = lf.leafi_select_leaves(idx, F)
    lf.leafi_set_filters(idx, fl, *lf.leafi_initial_weights(idx, F, M, 2502018361))
    Qg, Ql, _, _ = lf.leafi_training_queries(idx, lf.TrainParams(), fl)
    Tg = np.zeros((1500, F), np.float32)
    Tl = np.zeros((F, 500), np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lf.leafi_train_targets(idx, Qg, Ql, Tg, Tl)
    torch.cuda.synchronize()
    t_targets = time.perf_counter() - t0
    pairs = (1500 + 500) * float(sizes[fl].sum())
    t0 = time.perf_counter()
    enhance(idx, F, kclasses=(1, 10, 100), max_epochs=a.epochs, tune_search=int(a.tune))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    Q = fx.test_queries(X, a.queries)
    rng = np.random.default_rng(2504)
    ks = rng.choice([1, 10, 100], a.queries).astype(np.int32)
    tg = rng.choice([0.9, 0.95, 0.99], a.queries).astype(np.float64)
    Qd = torch.from_numpy(Q).cuda()
    kd = torch.from_numpy(ks).cuda()
    td = torch.from_numpy(tg).cuda()
    ids = torch.zeros((a.queries, 100), dtype=torch.int64, device="cuda")
    dd = torch.zeros((a.queries, 100), dtype=torch.float32, device="cuda")
    one = torch.ones_like(td)
    ex_i = torch.zeros_like(ids)
    ex_d = torch.zeros_like(dd)

    reps = max(1, a.steps // 30)

    def timed(targets, oi, od, tag):
        lf.leafi_search_mixed(idx, Qd, kd, targets, 100, oi, od)   # warm-up (graphs, buffers)
        torch.cuda.synchronize()
        st = lf.SearchStats()
        torch.cuda.nvtx.range_push(tag)
        t0 = time.perf_counter()
        for _ in range(reps):
            lf.leafi_search_mixed(idx, Qd, kd, targets, 100, oi, od, st)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        torch.cuda.nvtx.range_pop()
        return sec, st

    ms_ex, st_ex = timed(one, ex_i, ex_d, "timed_mixed_plain")
    ms_lf, st_lf = timed(td, ids, dd, "timed_mixed_leafi")
    lf.leafi_set_profiling(idx, 2)
    lf.leafi_search_mixed(idx, Qd, kd, td, 100, ids, dd)
    torch.cuda.synchronize()
    kt = lf.leafi_get_kernel_times(idx)
    lf.leafi_set_profiling(idx, 0)
    a_ids, e_ids = ids.cpu().numpy(), ex_i.cpu().numpy()
    rec = {}
    for kc in (1, 10, 100):
        for tv in (0.9, 0.95, 0.99):
            sel = np.where((ks == kc) & (tg == tv))[0]
            r = np.mean([len(set(a_ids[i, :kc]) & set(e_ids[i, :kc])) / kc for i in sel])
            rec["k%d_t%.2f" % (kc, tv)] = float(r)
    _emit({"metric": "mixed-k LeaFi-iSAX search: queries/s (and build-phase training targets)",
           "value": a.queries / ms_lf, "unit": "queries/s",
           "plain_lb_qps": a.queries / ms_ex, "recall_at_k_by_class": rec,
           "series_scanned_per_query": st_lf.series_scanned / a.queries,   # the last call's
           "plain_series_scanned_per_query": st_ex.series_scanned / a.queries,
           "waves_per_batch": st_lf.waves / max(1, st_lf.batches),
           "kernel_ms_per_search": {k: [v[0], v[1]] for k, v in kt.items() if v[1]},
           "training_targets": {"seconds": t_targets, "global_queries": 1500,
                                "local_queries_per_filter": 500, "filters": F,
                                "pairs": pairs, "tflops_fp16_equiv": pairs * 2 * M / t_targets / 1e12},
           "config": {"workload": "iSAX (16 segments, 8 bits) over %d random walks x %d, leaf "
                                  "capacity %d, %d queries, k in {1,10,100}, targets in "
                                  "{0.9,0.95,0.99}" % (a.n, M, a.leaf_cap, a.queries),
                      "leaves": info.n_leaves, "leaf_size_min_median_max":
                          [int(sizes.min()), float(np.median(sizes)), int(sizes.max())],
                      "filters": F, "scan_path": a.scan_path,
                      "wave": lf.leafi_get_info(idx).wave if a.tune else a.wave,
                      "wave_exact": lf.leafi_get_info(idx).wave_exact,
                      "tuned": bool(a.tune)},
           "build_s": {"data": t_data, "index": t_build, "train_and_tune": t_train},
           "data": "synthetic"})
    lf.leafi_free(idx)


def run_precision(a):
    """Embedding-like m = 96, k = 10 exact search: tensor-core scans (float16 or
    e4m3 products with per-series scales, float32 re-check band) vs CUDA-core
    scan, error against float64; and the flat contraction (one leaf holding
    every series) as the tensor-core case."""
    torch, lf = _gpu_setup()
    m, k = 96, 10
    t0 = time.perf_counter()
    X = fx.embedding_like(a.n, m)
    t_data = time.perf_counter() - t0
    Q = fx.test_queries(X, a.queries)
    Qd = torch.from_numpy(Q).cuda()
    out = {}
    res = {}
    for name, path, cap in (("tensor_core", 0, a.leaf_cap), ("cuda_core", 1, a.leaf_cap),
                            ("tensor_core_e4m3", 2, a.leaf_cap)):
        idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=cap, wave=a.wave, device=0,
                                               scan_path=path))
        ids = torch.zeros((a.queries, k), dtype=torch.int64, device="cuda")
        dd = torch.zeros((a.queries, k), dtype=torch.float32, device="cuda")
        lf.leafi_exact_search(idx, Qd, k, ids, dd)
        torch.cuda.synchronize()
        st = lf.SearchStats()
        reps = max(1, a.steps // 10)
        t0 = time.perf_counter()
        for _ in range(reps):
            lf.leafi_exact_search(idx, Qd, k, ids, dd, st)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        # the statistics describe the last call
        out[name] = {"qps": a.queries / sec, "series_scanned_per_query":
                     st.series_scanned / a.queries,
                     "rechecks_per_query": st.rechecks / a.queries,
                     "band_hit_rate": st.rechecks / max(1, st.series_scanned)}
        res[name] = (ids.cpu().numpy(), dd.cpu().numpy())
        lf.leafi_free(idx)
    same = bool(np.array_equal(res["tensor_core"][0], res["cuda_core"][0]) and
                np.array_equal(res["tensor_core"][1], res["cuda_core"][1]) and
                np.array_equal(res["tensor_core"][0], res["tensor_core_e4m3"][0]) and
                np.array_equal(res["tensor_core"][1], res["tensor_core_e4m3"][1]))
    # float64 reference on a sample: expanded-form distances rank candidates,
    # the top 4k are re-ranked with direct float64 differences
    rng = np.random.default_rng(2503)
    smp = np.sort(rng.choice(a.queries, 64, replace=False))
    X64 = X.astype(np.float64)
    Q64 = Q[smp].astype(np.float64)
    xx = np.einsum("ij,ij->i", X64, X64)
    d2 = np.empty((len(smp), a.n))
    for c0 in range(0, a.n, 1 << 20):
        c1 = min(a.n, c0 + (1 << 20))
        d2[:, c0:c1] = xx[c0:c1][None] - 2.0 * (Q64 @ X64[c0:c1].T)
    d2 += np.einsum("ij,ij->i", Q64, Q64)[:, None]
    cand = np.argpartition(d2, 4 * k, axis=1)[:, :4 * k]
    recall, max_rel = [], 0.0
    g_ids, g_d = res["tensor_core"]
    for j, qi in enumerate(smp):
        exact = np.sqrt(((X64[cand[j]] - Q64[j]) ** 2).sum(1))
        truth = cand[j][np.lexsort((cand[j], exact))[:k]]
        recall.append(len(set(g_ids[qi]) & set(truth)) / k)
        dg = np.sqrt(((X64[g_ids[qi]] - Q64[j]) ** 2).sum(1))
        max_rel = max(max_rel, float(np.max(np.abs(g_d[qi].astype(np.float64) - dg) / dg)))
    # flat contraction: one leaf with every series, 256 queries, all pairs
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=a.n, wave=1, device=0))
    lf.leafi_set_profiling(idx, 1)
    ids = torch.zeros((256, k), dtype=torch.int64, device="cuda")
    dd = torch.zeros((256, k), dtype=torch.float32, device="cuda")
    for _ in range(2):
        lf.leafi_exact_search(idx, Qd[:256], k, ids, dd)
    lf.leafi_set_profiling(idx, 1)
    reps = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        lf.leafi_exact_search(idx, Qd[:256], k, ids, dd)
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / reps
    kt = lf.leafi_get_kernel_times(idx)
    # every scan launch of a call (the route round holds all pairs; the next
    # round finds none) over the calls
    scan_ms = kt["leaf_scan"][0] / reps
    flops = 2.0 * 256 * a.n * m
    pk, pk_kind = peaks()
    tc_peak = pk.get("bf16_tflops", 1800.0)
    flat = {"qps": 256 / sec, "scan_ms_per_call": scan_ms,
            "scan_launches_per_call": kt["leaf_scan"][1] / reps,
            "achieved_tflops": flops / (scan_ms / 1e3) / 1e12, "peak_tflops": tc_peak,
            "frac": flops / (scan_ms / 1e3) / 1e12 / tc_peak,
            "peak_source": "fp16 dense = %s bf16 burst rate" % pk_kind,
            "algorithmic_flop_per_launch": flops}
    lf.leafi_free(idx)
    _emit({"metric": "precision path, k = 10: exact search queries/s and error against float64",
           "value": out["tensor_core"]["qps"], "unit": "queries/s", "paths": out,
           "all_paths_equal": same,
           "vs_float64": {"sample": len(smp), "max_rel_distance_error": max_rel,
                          "recall_at_10": float(np.mean(recall))},
           "flat_contraction": flat,
           "config": {"workload": "embedding-like (1,000 clusters, std 0.3) %d x %d, DSTree leaf "
                                  "capacity %d, %d queries, k = 10" % (a.n, m, a.leaf_cap, a.queries)},
           "build_s": {"data": t_data}, "data": "synthetic"})


def run_ablation(a):
    """Without local training data (Sec. 5, the -Local study): the batched
    random-walk workload searched exactly, with filters trained on global
    queries only (-Local) and on global plus local queries (+Local, LeaFi),
    recall target 0.99; throughput, series scanned and recall against exact."""
    torch, lf = _gpu_setup()
    from paper_2502_01836_b300.workflow import enhance
    X = fx.random_walk(a.n, M)
    Q = fx.test_queries(X, a.queries)
    Qd = torch.from_numpy(Q).cuda()
    ids = torch.zeros((a.queries, 1), dtype=torch.int64, device="cuda")
    dd = torch.zeros((a.queries, 1), dtype=torch.float32, device="cuda")

    def timed(idx, target):
        for _ in range(a.warmup):
            lf.leafi_search(idx, Qd, 1, target, ids, dd)
        st = lf.SearchStats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(1, a.steps // 3)
        for _ in range(reps):
            lf.leafi_search(idx, Qd, 1, target, ids, dd, st)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        return a.queries / sec, ids[:, 0].cpu().numpy().copy(), st.series_scanned / a.queries

    rows = {}
    bp = lf.BuildParams(leaf_capacity=a.leaf_cap, wave=a.wave, device=0)
    idx = lf.leafi_build(X, bp)
    qps, exact, ser = timed(idx, 1.0)
    rows["exact"] = {"qps": qps, "series_scanned_per_query": ser, "recall_at_1": 1.0}
    lf.leafi_free(idx)
    # -Local: the 1,500 global queries only; +Local: 500 local queries per filter added
    for name, (n_train, ratio) in (("-Local", (1500, float("inf"))), ("+Local", (2000, 3.0))):
        idx = lf.leafi_build(X, bp)
        enhance(idx, a.filters, n_train=n_train, global_local_ratio=ratio, max_epochs=a.epochs,
                tune_search=int(a.tune))
        qps, got, ser = timed(idx, a.target)
        rows[name] = {"qps": qps, "series_scanned_per_query": ser,
                      "recall_at_1": float(np.mean(got == exact)),
                      "meets_target": bool(np.mean(got == exact) >= a.target)}
        lf.leafi_free(idx)
    _emit({"metric": "LeaFi without and with local training data: queries/s and recall@1",
           "unit": "queries/s", "value": rows["+Local"]["qps"], "rows": rows,
           "config": {"workload": "DSTree over %d random walks x %d, leaf capacity %d, filters on "
                                  "the %d largest leaves, %d queries, 1-NN, target %.2f, wave %d"
                                  % (a.n, M, a.leaf_cap, a.filters, a.queries, a.target, a.wave)},
           "data": "synthetic"})


def run_cnn(a):
    """The model-type study (Sec. 5.2, Table 1): MLP and CNN filters (two k = 3
    convolutions with C = m channels) on the embedding-like series of length 96
    that stand in for Deep; for each model, Alg. 3's measured t^F and
    threshold th, then filters on the a.filters largest leaves: training time,
    queries/s, recall@1 and series scanned at the recall target, beside exact
    search."""
    torch, lf = _gpu_setup()
    from paper_2502_01836_b300.workflow import enhance
    m = 96
    X = fx.embedding_like(a.n, m)
    Q = fx.test_queries(X, a.queries)
    Qd = torch.from_numpy(Q).cuda()
    ids = torch.zeros((a.queries, 1), dtype=torch.int64, device="cuda")
    dd = torch.zeros((a.queries, 1), dtype=torch.float32, device="cuda")

    def timed(idx, target):
        for _ in range(a.warmup):
            lf.leafi_search(idx, Qd, 1, target, ids, dd)
        st = lf.SearchStats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = max(1, a.steps // 3)
        for _ in range(reps):
            lf.leafi_search(idx, Qd, 1, target, ids, dd, st)
        torch.cuda.synchronize()
        sec = (time.perf_counter() - t0) / reps
        # the statistics describe the last call
        return a.queries / sec, ids[:, 0].cpu().numpy().copy(), st.series_scanned / a.queries

    bp = lf.BuildParams(leaf_capacity=a.leaf_cap, wave=a.wave, device=0)
    idx = lf.leafi_build(X, bp)
    L = lf.leafi_get_info(idx).n_leaves
    qps, exact, ser = timed(idx, 1.0)
    rows = {"exact": {"qps": qps, "series_scanned_per_query": ser, "recall_at_1": 1.0}}
    for name, model in (("MLP", lf.FILTER_MLP), ("CNN", lf.FILTER_CNN)):
        sel, rep = lf.leafi_select_leaves_auto(idx, a=2.0, model=model)
        t0 = time.perf_counter()
        enh = enhance(idx, a.filters, max_epochs=a.epochs, tune_search=int(a.tune), model=model)
        t_train = time.perf_counter() - t0
        qps, got, ser = timed(idx, a.target)
        rec = float(np.mean(got == exact))
        rows[name] = {"alg3": {"t_filter_s": rep["t_filter_s"], "t_series_s": rep["t_series_s"],
                               "threshold": rep["threshold"], "n_selected": rep["n_selected"]},
                      "train_and_tune_s": t_train,
                      "epochs_run_mean": float(np.mean(enh.epochs_run)),
                      "qps": qps, "series_scanned_per_query": ser, "recall_at_1": rec,
                      "meets_target": bool(rec >= a.target),
                      "wave": lf.leafi_get_info(idx).wave}
    lf.leafi_free(idx)
    _emit({"metric": "filter model study: queries/s, recall@1 and Alg. 3 threshold, MLP vs CNN",
           "unit": "queries/s", "value": rows["CNN"]["qps"], "rows": rows,
           "config": {"workload": "DSTree over %d embedding-like series x %d (1,000 clusters, "
                                  "std 0.3), leaf capacity %d (%d leaves), filters on the %d "
                                  "largest leaves, %d queries, 1-NN, target %.2f"
                                  % (a.n, m, a.leaf_cap, L, a.filters, a.queries, a.target)},
           "data": "synthetic"})


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.config != "batched":
        {"serving": run_serving, "mixed": run_mixed, "precision": run_precision,
         "ablation": run_ablation, "cnn": run_cnn}[a.config](a)
        return
    import torch
    rank, world, local, dist = dist_setup(a.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2502_01836_b300 as lf
    from paper_2502_01836_b300.workflow import enhance

    X = fx.random_walk(a.n, M)
    idx = lf.leafi_build(X, lf.BuildParams(leaf_capacity=a.leaf_cap, wave=a.wave, device=local,
                                           scan_path=a.scan_path))
    stream = torch.cuda.current_stream(dev)
    lf.leafi_set_stream(idx, stream.cuda_stream)
    lf.leafi_set_query_schedule(idx, not a.no_schedule)
    lf.leafi_set_search_lanes(idx, a.lanes)
    lf.leafi_set_search_batch(idx, a.batch or a.launch)
    lf.leafi_set_scan_part(idx, a.part, a.items_per_sm, a.min_part, a.scan_blocks)
    t_train = time.perf_counter()
    enh = enhance(idx, a.filters, kclasses=(1,), max_epochs=a.epochs, tune_search=int(a.tune))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t_train
    info = lf.leafi_get_info(idx)
    Q = fx.test_queries(X, a.queries, seed=fx.SEED_TEST + 1000 * rank)
    Qd = torch.from_numpy(Q).to(dev)
    nl = (a.queries + a.launch - 1) // a.launch
    ids = torch.empty((a.queries, 1), dtype=torch.int64, device=dev)
    dd = torch.empty((a.queries, 1), dtype=torch.float32, device=dev)
    ex_ids = torch.empty_like(ids)
    ex_d = torch.empty_like(dd)

    def run(target, out_i, out_d, lat=None, stats=None, per_launch=False):
        # one call over all queries (the library runs them in launches of
        # a.launch, several in flight), or one call per launch for the latencies
        spans = ([(b * a.launch, min(a.queries, (b + 1) * a.launch)) for b in range(nl)]
                 if per_launch else [(0, a.queries)])
        for s0, s1 in spans:
            st = lf.SearchStats()
            if lat is not None:
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            lf.leafi_search(idx, Qd[s0:s1], 1, target, out_i[s0:s1], out_d[s0:s1], st)
            if lat is not None:
                e1.record(stream)
                lat.append((e0, e1))
            if stats is not None:
                for f, _ in lf.SearchStats._fields_:
                    stats[f] = stats.get(f, 0) + getattr(st, f)

    def timed(target, out_i, out_d, profile=False):
        ck = Clocks(local).__enter__()   # sampling starts before the warm-up
        for _ in range(a.warmup):
            run(target, out_i, out_d)
        if profile:
            lf.leafi_set_profiling(idx, 1)   # leaf-scan launches only: the cheapest level
        lat, stats = [], {}
        barrier(dist)
        torch.cuda.synchronize()
        launches0 = lf.leafi_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_leafi" if target < 1.0 else "timed_plain")
        t_0 = time.perf_counter()
        e0.record(stream)
        for _ in range(a.steps):
            run(target, out_i, out_d, None, stats)
        e1.record(stream)
        torch.cuda.synchronize()
        t_1 = time.perf_counter()
        torch.cuda.nvtx.range_pop()
        time.sleep(0.15)
        ck.__exit__()
        ck.mark(t_0, t_1)
        barrier(dist)
        launches = lf.leafi_launch_count() - launches0
        ms = e0.elapsed_time(e1) / a.steps
        kt = lf.leafi_get_kernel_times(idx) if profile else None
        if profile:
            lf.leafi_set_profiling(idx, 0)
        # latency of one launch-sized call (a request of a.launch queries), untimed pass
        run(target, out_i, out_d, lat, None, per_launch=True)
        torch.cuda.synchronize()
        lats = [x.elapsed_time(y) for x, y in lat]
        return ms, lats, stats, launches, ck.summary(), kt

    pk0, _ = peaks()
    # exact (plain-bound) search: ground truth and the comparison arm
    ms_ex, lat_ex, st_ex, _, _, _ = timed(1.0, ex_ids, ex_d)
    ms, lat, st, launches, clocks, kt = timed(a.target, ids, dd, profile=False)
    # the scan alone: the same steps with one lane (batches one after another,
    # so no scan launch waits for SMs held by another lane's), every leaf-scan
    # launch timed with CUDA events on the lane stream it runs on
    lf.leafi_set_search_lanes(idx, 1)
    run(a.target, ids, dd)
    lf.leafi_set_profiling(idx, 1)
    ser_stats = {}
    torch.cuda.synchronize()
    e0s = torch.cuda.Event(enable_timing=True)
    e1s = torch.cuda.Event(enable_timing=True)
    ser_steps = max(3, a.steps // 4)
    e0s.record(stream)
    for _ in range(ser_steps):
        run(a.target, ids, dd, None, ser_stats)
    e1s.record(stream)
    torch.cuda.synchronize()
    ser_ms = e0s.elapsed_time(e1s) / ser_steps
    kt = lf.leafi_get_kernel_times(idx)
    # one more one-lane step with the scan's in-kernel launch timeline
    lf.leafi_set_profiling(idx, 2)
    run(a.target, ids, dd)
    torch.cuda.synchronize()
    ph1 = lf.leafi_get_scan_phases(idx)
    lf.leafi_set_profiling(idx, 0)
    lf.leafi_set_search_lanes(idx, a.lanes)
    nl1 = max(ph1["launches"], 1)
    timeline = {"launches": ph1["launches"],
                "span_us": ph1["launch_span_ns"] / nl1 / 1e3,
                "start_skew_us": ph1["start_skew_ns"] / nl1 / 1e3,
                "end_skew_us": ph1["end_skew_ns"] / nl1 / 1e3,
                "block_resident_us": ph1["epilogue_span"] / SMS / nl1 / (pk0.get("sm_max_mhz", 2032.0))}
    # Alg. 3 with this device's costs (the run above uses the configuration's
    # 100 largest leaves, i.e. th = 0)
    sel_fl, sel_rep = lf.leafi_select_leaves_auto(idx, a=2.0, mem_cap=8 << 30)
    # per-kind breakdown and scan phase counters from one more (untimed) step
    lf.leafi_set_profiling(idx, 2)
    run(a.target, ids, dd)
    torch.cuda.synchronize()
    kt_all = lf.leafi_get_kernel_times(idx)
    kt_all["_phases"] = lf.leafi_get_scan_phases(idx)
    lf.leafi_set_profiling(idx, 0)
    recall = float((ids[:, 0] == ex_ids[:, 0]).float().mean().item())
    ms_max = max_over_ranks(ms, dist, dev)
    ms_ex_max = max_over_ranks(ms_ex, dist, dev)
    value = world * a.queries / (ms_max / 1e3)
    value_ex = world * a.queries / (ms_ex_max / 1e3)

    # end to end through the public API with pinned host buffers (the copies run
    # inside the timed region, overlapped with the other lane's work)
    Qh = torch.from_numpy(Q).pin_memory()
    ih = torch.zeros((a.queries, 1), dtype=torch.int64).pin_memory()
    dh = torch.zeros((a.queries, 1), dtype=torch.float32).pin_memory()
    lf.leafi_search(idx, Qh, 1, a.target, ih, dh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        lf.leafi_search(idx, Qh, 1, a.target, ih, dh)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / a.steps, dist, dev)
    e2e = {"value": world * a.queries / (e2e_ms / 1e3), "unit": "queries/s",
           "h2d_bytes_per_step": a.queries * M * 4, "d2h_bytes_per_step": a.queries * (8 + 4)}

    # roofline of the dominant kernel (leaf scan).  Algorithmic bytes per launch:
    # the series of the distinct leaves each scan round reads x the bytes of one
    # scanned row (float16 rows of kp halves on the tensor-core path).  Duration:
    # the mean CUDA-event time of the leaf-scan launches in the serialised pass.
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6400.0)
    clk = pk.get("sm_max_mhz", 2032.0)
    scan_ms, scan_n = kt["leaf_scan"]
    scan_launch_ms = scan_ms / max(scan_n, 1)
    bytes_launch = ser_stats["distinct_series"] * info.scan_row_bytes / max(scan_n, 1)
    pairs_launch = ser_stats["series_scanned"] / max(scan_n, 1)
    achieved_gbs = bytes_launch / (scan_launch_ms / 1e3) / 1e9
    roof_hbm = achieved_gbs / hbm
    # the whole timed (eight-lane) step charged to the scan: a lower bound
    step_bytes = st["distinct_series"] / a.steps * info.scan_row_bytes
    step_view = {"achieved_gbs": step_bytes / (ms / 1e3) / 1e9,
                 "frac": step_bytes / (ms / 1e3) / 1e9 / hbm,
                 "bytes_per_step": step_bytes, "ms_per_step": ms}
    cross = {"scan_ms_per_step": scan_ms / ser_steps, "serialised_ms_per_step": ser_ms,
             "scan_share": scan_ms / ser_steps / ser_ms}
    traffic, traffic_src = None, None
    try:
        src = os.path.join(ROOT, "paper_2502_01836_b300", "csrc", "k_scan_tc.cu")
        same_kernel = code_sha1(src, "__global__ void round_prep_kernel(") == \
            SCAN_TRAFFIC["kernel_sha1"]
        default_workload = (a.n, a.leaf_cap, a.filters, a.launch, a.wave) == \
            (1_000_000, 10_000, 100, 256, 64)
        if info.tensor_scan and same_kernel and default_workload:
            traffic = SCAN_TRAFFIC["bytes_per_launch"]
            traffic_src = SCAN_TRAFFIC["source"]
    except OSError:
        pass
    if info.tensor_scan:
        tc_tf = pairs_launch * 2.0 * M / (scan_launch_ms / 1e3) / 1e12
        tc_peak = pk.get("bf16_tflops", 1800.0)
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": roof_hbm, "traffic": traffic, "traffic_source": traffic_src,
                    "peak_source": pk_kind, "bytes_per_launch": bytes_launch,
                    "launch_ms": scan_launch_ms,
                    "measured": "leaf-scan launches of %d one-lane steps (serialised), CUDA "
                                "events on the launching stream" % ser_steps,
                    "tensor_view": {"achieved_tflops": tc_tf, "peak": tc_peak,
                                    "frac": tc_tf / tc_peak,
                                    "peak_source": "fp16 dense = measured bf16 burst rate"}}
    else:
        alu_peak = SMS * FP32_LANES * clk * 1e6 * 1.5 / 1e12   # FSUB+FFMA: 3 FLOP per 2 instr
        achieved_tf = pairs_launch * M * 3.0 / (scan_launch_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved_tf / alu_peak, "traffic": None,
                    "peak_source": "148 SMs x 128 FP32 lanes x %.0f MHz x 1.5 FLOP/instr (%s clocks)"
                                   % (clk, pk_kind),
                    "hbm_view": {"achieved_gbs": achieved_gbs, "frac": roof_hbm}}
    roofline["kernel"] = "leaf_scan (tensor cores)" if info.tensor_scan else "leaf_scan (CUDA cores)"
    roofline["step_view"] = step_view
    roofline["cross_check"] = cross
    roofline["timeline_one_lane"] = timeline
    roofline["bytes_per_series"] = info.scan_row_bytes
    span = kt_all.get("_phases", {}).get("epilogue_span", 0.0)
    if info.tensor_scan and span > 0:
        # the same bytes over the time a CTA is resident (per-SM cycle counter of
        # the profiled eight-lane step)
        resident_s = span / SMS / (clock_mhz(clocks, clk) * 1e6)
        distinct = st["distinct_series"] / a.steps
        roofline["resident_view"] = {"achieved_gbs": distinct * info.scan_row_bytes / resident_s / 1e9,
                                     "frac": distinct * info.scan_row_bytes / resident_s / 1e9 / hbm,
                                     "resident_ms_per_step": resident_s * 1e3}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        try:
            W = (np.zeros((a.filters, M, M), np.float32), np.zeros((a.filters, M), np.float32),
                 np.zeros((a.filters, M), np.float32), np.zeros(a.filters, np.float32))
            lf.leafi_get_filters(idx, *W)
            alpha = np.zeros((a.filters, info.n_calib))
            qp = np.zeros((1, info.n_calib))
            lf.leafi_get_autotuners(idx, alpha, qp)
            rate, dt, _ = oracle_leafi_rate(X, enh.filter_leaf, W, alpha, qp[0], Q, a.leaf_cap,
                                            info.wave, a.target, a.cpu_sample)
            cpu = {"value": rate, "unit": "queries/s", "cores": cpu_threads(), "kind": "oracle",
                   "sample": "%d of the %d queries, LeaFi search with the same filters and "
                             "auto-tuner tables (%.1f s)" % (a.cpu_sample, a.queries, dt)}
        except Exception as e:  # reported, never fatal
            cpu = {"value": None, "unit": "queries/s", "cores": cpu_threads(), "kind": "oracle",
                   "sample": "failed: %s" % e}

    if rank == 0:
        lat_sorted = sorted(lat)
        line = {
            "metric": "queries/s at 99% recall (LeaFi search)", "value": value,
            "unit": "queries/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(a),
            "recall_at_1": recall,
            "plain_lb": {"value": value_ex, "unit": "queries/s", "ms_per_step": ms_ex_max,
                         "series_scanned_per_query": st_ex["series_scanned"] / (a.steps * a.queries),
                         "distinct_bytes_per_batch": st_ex["distinct_series"] * info.scan_row_bytes
                                                     / max(st_ex["batches"], 1),
                         "p50_ms": float(np.percentile(lat_ex, 50)),
                         "p99_ms": float(np.percentile(lat_ex, 99))},
            "speedup_vs_plain_lb": value / value_ex,
            "latency_per_launch_ms": {"p50": float(np.percentile(lat_sorted, 50)),
                                      "p99": float(np.percentile(lat_sorted, 99))},
            "series_scanned_per_query": st["series_scanned"] / (a.steps * a.queries),
            # bytes of the distinct series a batch's rounds read (a series read in two
            # rounds counts twice), LeaFi here and plain-LB above
            "distinct_bytes_per_batch": st["distinct_series"] * info.scan_row_bytes
                                        / max(st["batches"], 1),
            "rechecks_per_query": st["rechecks"] / (a.steps * a.queries),
            "pruning_ratio": 1.0 - st["series_scanned"] / (a.steps * a.queries * a.n),
            # per query: leaves pruned by the summarisation bound and by a filter (Alg. 2)
            "leaves_per_query": {"searched": st["leaves_scanned"] / (a.steps * a.queries),
                                 "bound_pruned": st["lb_pruned"] / (a.steps * a.queries),
                                 "filter_pruned": st["filter_pruned"] / (a.steps * a.queries),
                                 "plain_searched": st_ex["leaves_scanned"] / (a.steps * a.queries)},
            # filter predictions made per query (query tiles whose pairs no wave
            # select can read are skipped once the route leaves set a best-so-far)
            "filter_evals_per_query": st["filter_evals"] / (a.steps * a.queries),
            "plain_pruning_ratio": 1.0 - st_ex["series_scanned"] / (a.steps * a.queries * a.n),
            "waves_per_launch": st["waves"] / max(st["batches"], 1),
            "host_ms_per_step": {"call": st["host_ms"] / a.steps,
                                 "waiting_for_gpu": st["host_wait_ms"] / a.steps,
                                 "busy": (st["host_ms"] - st["host_wait_ms"]) / a.steps},
            "graph_batch_fraction": st["graph_batches"] / max(st["batches"], 1),
            "leaf_selection_alg3": dict(sel_rep, a=2.0, mem_cap_bytes=8 << 30),
            "kernel_ms_per_step": {k: v[0] for k, v in kt_all.items()
                                   if not k.startswith("_") and v[1]},
            "kernel_ms_note": "one extra untimed step with every kind timed",
            "scan_phase_cycles_per_block": {k: v / SMS for k, v in kt_all["_phases"].items()
                                            if not k.endswith("_ns") and k != "launches"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
            "build": {"leaves": info.n_leaves, "filters": info.n_filters,
                      "wave": info.wave, "wave_exact": info.wave_exact,
                      "items_per_sm": info.items_per_sm,
                      "train_and_tune_s": t_train,
                      "epochs_run_mean": float(np.mean(enh.epochs_run))},
        }
        print(json.dumps(line), flush=True)
    lf.leafi_free(idx)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
