#!/usr/bin/env python3
"""Benchmark of the sparse Sinkhorn-Knopp WMD on GB300.

One step = one query against the whole resident corpus: the cdist/K build
(K1) and the fused SDDMM+SpMM loop with the final reduction (K2+K3), i.e. all
N WMD values for the paper-shaped workload (V=100000, d=300, N=5000
documents of 20-150 Zipf(1.1) words, v_r=30, lambda=10, max_iter=15).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the host cores instead (the reference arm; there is no runnable
reference implementation of the paper).  Multi-GPU runs (torchrun) are
independent replicas: every rank answers the same query stream against its
own copy of the corpus, with no data-path collective.
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

from paper_2005_06727_gb300 import synth  # noqa: E402

METRIC = "query x doc WMDs/sec @15 iters, HBM GB/s % of peak; served p50/p99 latency"
UNIT = "WMDs/s"
L2_FLUSH_BYTES = 512 << 20
FP32_LANES_PER_SM = 128
WORKLOADS = {"paper": synth.PAPER, "tiny": synth.TINY, "large": synth.LARGE}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="paper")
    ap.add_argument("--prec", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--legs", default="converge,topk,dense,large,paper_exact,batched,serving",
                    help="comma-separated extra legs to run after the timed step")
    ap.add_argument("--no-systems", action="store_true",
                    help="skip the batched and served measurements")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="Poisson requests per offered rate (a fifth of them at 0.1x capacity)")
    ap.add_argument("--serving-workload", choices=["paper", "serving"], default="serving",
                    help="corpus of the serving leg: the full serving configuration (default, "
                         "V = N = 200,000) or the paper-shaped one")
    ap.add_argument("--shard-docs", action="store_true",
                    help="under torchrun: split the corpus's documents across the ranks "
                         "(nnz-balanced) and gather the WMD slices every step, instead of "
                         "independent replicas")
    ap.add_argument("--loop-variant", type=int, default=-1,
                    help="fused-loop tile variant (default: chosen by the autotuner)")
    ap.add_argument("--loop-partition", type=int, default=100,
                    help="team-size fill of the pinned --loop-variant (50, 75, 100, 200)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def replica_throughput(step_ms: float, units_per_rank: int, world: int, group=None):
    """Whole-job throughput of independent replicas: every rank processed
    `units_per_rank` units; the job takes as long as the slowest rank.
    Returns (value, max step ms over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(step_ms)], dtype=torch.float64)
    if world > 1:
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    worst = float(t.item())
    return world * units_per_rank / (worst * 1e-3), worst


def workload_name(w):
    return (f"{w.name}: V={w.V} d={w.d} N={w.N} docs of {w.doc_lo}-{w.doc_hi} Zipf(1.1) words, "
            f"v_r={w.vr_lo}, lambda={w.lam:g}, max_iter={w.max_iter}")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def recorded_traffic(kernel: str, workload: str, loop_variant=None, loop_partition=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    this workload (and loop variant and partition) and the kernel's source is
    unchanged since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("workload") != workload:
        return None
    if loop_variant is not None and rec.get("loop_variant") != loop_variant:
        return None
    if loop_partition is not None and rec.get("loop_partition", 100) != loop_partition:
        return None
    src = os.path.join(ROOT, "paper_2005_06727_gb300", "csrc", rec["source"])
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    return rec["bytes_per_launch"] if sha == rec["source_sha256"] else None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ oracle
def time_oracle(w, vecs, c, q_ids, q_w, docs=None):
    from oracle import sinkhorn_wmd as orc
    t0 = time.perf_counter()
    out = orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N, vecs, w.lam,
                                  w.max_iter, docs=docs)
    return time.perf_counter() - t0, out


SAMPLE_ABOVE = 20_000   # corpora above this many documents: the oracle runs on a sample


def oracle_docs(c, n_sample=2000, seed=0):
    """All documents, or for large corpora a seeded sample that includes the
    20 longest and 20 shortest."""
    if c.N <= SAMPLE_ABOVE:
        return None
    rng = np.random.default_rng(seed)
    lens = np.diff(c.doc_ptr)
    return np.unique(np.concatenate([rng.choice(c.N, n_sample, replace=False),
                                     np.argsort(lens)[-20:], np.argsort(lens)[:20]]))


def cpu_baseline(w, vecs, c, q_ids, q_w, budget_s=10.0):
    """The oracle as it stands on the bench query, repeated until ~budget_s:
    whole queries, or a document sample on large corpora (the oracle's time
    per query grows with the documents it covers).  Returns the baseline
    record, the sampled document ids (None: all) and the oracle's WMDs."""
    docs = oracle_docs(c)
    n = c.N if docs is None else docs.size
    times = []
    ref = None
    while sum(times) < budget_s and len(times) < 5:
        t, ref = time_oracle(w, vecs, c, q_ids, q_w, docs=docs)
        times.append(t)
    t = statistics.mean(times)
    what = (f"all {w.N} documents" if docs is None else
            f"{n} of {w.N} documents (seeded sample incl. the 20 longest and 20 shortest)")
    return {"value": n / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} runs of the bench query over {what}, v_r={len(q_ids)}, "
                      f"FP64 numpy/scipy oracle, single thread, mean {t:.2f} s per run"}, docs, ref


_ORACLE_WORKER = {}


def _oracle_worker_init(cfg: int, root: str):
    """Pool initializer: rebuild the seeded workload in the worker (cheaper
    than shipping the arrays, and the same bits)."""
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_2005_06727_gb300 import synth as s
    w = s.WORKLOADS[cfg]
    vecs, c, qs = s.make_workload(w, 1)
    _ORACLE_WORKER.update(w=w, vecs=vecs, c=c, q=qs[0])


def _oracle_worker_run(docs):
    from oracle import sinkhorn_wmd as orc
    st = _ORACLE_WORKER
    w, c = st["w"], st["c"]
    t0 = time.perf_counter()
    orc.sinkhorn_wmd_sparse(st["q"][0], st["q"][1], c.row_ptr, c.doc_idx, c.val, c.N, st["vecs"],
                            w.lam, w.max_iter, docs=np.asarray(docs))
    return time.perf_counter() - t0


def cpu_baseline_all_cores(w, c, docs=None, timeout_s=300.0):
    """The same oracle on every host core: the documents (all, or the sample
    of a large corpus) split into one slice per core, each slice run by a
    single-threaded worker process (spawned: the parent already holds a CUDA
    context), timed from the first slice's start to the last one's end."""
    import concurrent.futures as cf
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ids = np.arange(c.N) if docs is None else np.asarray(docs)
    chunks = [ch for ch in np.array_split(ids, n) if ch.size]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        # an executor (not multiprocessing.Pool): a worker that cannot start
        # raises BrokenProcessPool instead of being respawned for ever
        with cf.ProcessPoolExecutor(len(chunks), mp_context=mp.get_context("spawn"),
                                    initializer=_oracle_worker_init,
                                    initargs=(w.cfg, ROOT)) as pool:
            list(pool.map(_oracle_worker_run, [ch[:4] for ch in chunks], timeout=timeout_s))
            t0 = time.perf_counter()
            list(pool.map(_oracle_worker_run, chunks, timeout=timeout_s))
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    what = f"all {c.N} documents" if docs is None else f"{ids.size} of {c.N} documents (seeded sample)"
    return {"value": ids.size / wall, "unit": UNIT, "cores": len(chunks), "kind": "oracle",
            "sample": f"the bench query over {what}, split into {len(chunks)} slices run by "
                      f"single-threaded worker processes at once, FP64 numpy/scipy oracle, "
                      f"{wall:.2f} s wall"}


def error_vs_oracle(got, ref, prec):
    """Largest per-document relative error of the GPU result against the FP64
    oracle (absolute floor 1e-7), beside the tolerance the tests enforce."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    ok = ~np.isnan(ref)
    rel = np.abs(got[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), 1e-7)
    nan_mismatch = int(np.sum(np.isnan(got) != np.isnan(ref)))
    return {"max_rel": float(np.max(rel)) if rel.size else 0.0,
            "mean_rel": float(np.mean(rel)) if rel.size else 0.0, "docs": int(ref.size),
            "nan_mismatch": nan_mismatch,
            "tolerance": 1e-5 if prec == wmd_prec_fp32() else 5e-3}


def wmd_prec_fp32():
    from paper_2005_06727_gb300 import wmd
    return wmd.PREC_FP32


def effective_hbm(w, c, v_r, loop_ms, step_ms, peak_gbs):
    """The paper's per-iteration formulation streams c and the dense u/x
    state in every SDDMM_SpMM pass and reads K and M once:
    B_iter = (T+1) [8 nnz + 4 (N+1) + 8 v_r N] + 4 v_r V 2 + 8 N bytes.
    Its bytes over the measured time, as a fraction of the HBM peak."""
    T = w.max_iter
    b_iter = (T + 1) * (8 * c.nnz + 4 * (c.N + 1) + 8 * v_r * c.N) + 4 * v_r * w.V * 2 + 8 * c.N
    loop_gbs = b_iter / (loop_ms * 1e-3) / 1e9
    step_gbs = b_iter / (step_ms * 1e-3) / 1e9
    return {"b_iter_bytes": int(b_iter), "loop_gbs": loop_gbs, "loop_frac": loop_gbs / peak_gbs,
            "step_gbs": step_gbs, "step_frac": step_gbs / peak_gbs, "peak_gbs": peak_gbs,
            "note": "B_iter of the paper's per-iteration formulation over the fused loop's (and "
                    "the whole step's) time; the loop itself is bound by FP32 ALUs (see roofline)"}


def run_reference(args, w):
    rank, _, world = dist_env()
    if rank != 0:
        return
    vecs, c, qs = synth.make_workload(w)
    q_ids, q_w = qs[0]
    # each step: one whole query (all documents), as the GPU arm's step; about
    # 1.7 s on a Grace core, so the default run stays well within a few minutes
    # (large corpora: a seeded document sample per step, see oracle_docs)
    docs = oracle_docs(c)
    n = c.N if docs is None else docs.size
    steps = []
    for k in range(args.warmup + args.steps):
        t, _ = time_oracle(w, vecs, c, q_ids, q_w, docs=docs)
        if k >= args.warmup:
            steps.append(t)
    t = statistics.mean(steps)
    value = n / t
    what = f"all {c.N} documents" if docs is None else f"a seeded sample of {n} of {c.N} documents"
    sample = (f"one query per step over {what}, v_r={len(q_ids)}, FP64 "
              f"numpy/scipy oracle, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(w), "impl": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ batched and served
def autotune_classes(corpus, qs, w):
    """Autotune every width class of the fused loop that one of the queries
    qs falls in (with the first such query), untimed."""
    from paper_2005_06727_gb300 import wmd as _w
    seen = set()
    for q in qs:
        width = _w.loop_width(len(q[0]))
        if width not in seen:
            seen.add(width)
            corpus.autotune(q[0], q[1], w.lam, w.max_iter)


def bench_batched(wmd, device, reps=2, with_oracle=True):
    """256 queries of v_r ~ U[5,128] against N=20000 documents: one at a time
    through wmd_query versus one wmd_query_batch call (graph replayed)."""
    wb = synth.BATCHED
    vecs, c, qs = synth.make_workload(wb)
    corpus = wmd.Corpus.from_synth(vecs, c, device=device)
    autotune_classes(corpus, qs, wb)  # every width class the batch uses
    out = np.empty(c.N, np.float64)
    for q in qs[:4]:
        corpus.query(q[0], q[1], wb.lam, wb.max_iter, out=out)
    t0 = time.perf_counter()
    for q in qs:
        corpus.query(q[0], q[1], wb.lam, wb.max_iter, out=out)
    t_single = time.perf_counter() - t0
    corpus.query_batch(qs, wb.lam, wb.max_iter)  # first call runs eagerly and captures
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        res = corpus.query_batch(qs, wb.lam, wb.max_iter)
        times.append(time.perf_counter() - t0)
    t_batch = min(times)
    assert np.array_equal(res[-1], out), "batched and single results differ"
    units = len(qs) * c.N
    corpus.close()
    rec = {"workload": (f"{wb.name}: V={wb.V} d={wb.d} N={wb.N} docs of {wb.doc_lo}-{wb.doc_hi} "
                        f"words, {len(qs)} queries v_r U[{wb.vr_lo},{wb.vr_hi}], lambda={wb.lam:g}, "
                        f"max_iter={wb.max_iter}"),
           "one_at_a_time": {"value": units / t_single, "unit": UNIT, "seconds": t_single},
           "batched": {"value": units / t_batch, "unit": UNIT, "seconds": t_batch,
                       "path": "wmd_query_batch (captured CUDA graph replay)"},
           "speedup": t_single / t_batch}
    if with_oracle:
        # every query of the batch against the FP64 oracle on a document
        # sample (after the timing: the workers load the host cores)
        rec["error_vs_oracle"] = batch_errors_vs_oracle(wb, c, qs, res)
    return rec


def batch_errors_vs_oracle(w, c, qs, res, n_docs=200):
    """Largest relative error over every query of a batch, each against the
    FP64 oracle on the same seeded sample of documents (the 20 longest and
    shortest included), run in spawned single-threaded workers."""
    from oracle.pool import OraclePool, sample_documents
    docs = sample_documents(c.doc_ptr, n_docs)
    worst, worst_q = 0.0, -1
    t0 = time.perf_counter()
    with OraclePool(w.cfg) as pool:
        futs = [pool.submit(q[0], q[1], w.lam, w.max_iter, docs) for q in qs]
        for k, f in enumerate(futs):
            ref, _ = f.result(timeout=3600)
            e = error_vs_oracle(res[k][docs], ref, wmd_prec_fp32())
            if e["max_rel"] > worst:
                worst, worst_q = e["max_rel"], k
        workers = pool.workers
    return {"max_rel": worst, "worst_query": worst_q, "queries": len(qs), "documents": int(docs.size),
            "tolerance": 1e-5, "oracle_workers": workers, "oracle_wall_s": time.perf_counter() - t0,
            "sample": f"every query on {docs.size} seeded documents (20 longest and 20 shortest included)"}


def bench_serving(wmd, device, n_requests=2000, seed=11, workload="serving", n_checked=16):
    """Poisson arrivals (v_r ~ U[5,200]) against the full serving corpus (or
    the paper-shaped one): latency p50/p99 and throughput of the
    continuous-batching server at 0.1x to 1.2x of its measured capacity, the
    one-query-at-a-time capacity, and the served results of n_checked
    distinct queries (v_r = 200 among them) against the FP64 oracle."""
    import threading as th
    w = synth.SERVING if workload == "serving" else synth.PAPER
    vecs, c, _ = synth.make_workload(w, 0)
    corpus = wmd.Corpus.from_synth(vecs, c, device=device)
    rng = np.random.default_rng(seed)
    qs = [synth.make_query(w.V, 200 if i == 0 else int(rng.integers(5, 201)), 50_000 + i)
          for i in range(64)]
    served = {}   # query index -> its first served result (n_checked distinct queries)
    autotune_classes(corpus, qs, w)
    out = np.empty(c.N, np.float64)
    for q in qs[:4]:
        corpus.query(q[0], q[1], w.lam, w.max_iter, out=out)
    t0 = time.perf_counter()
    for q in qs:
        corpus.query(q[0], q[1], w.lam, w.max_iter, out=out)
    single_qps = len(qs) / (time.perf_counter() - t0)

    srv = wmd.Server(corpus, max_batch=32, slots=3, mem_budget=24 << 30)
    try:
        # capacity: a closed burst of requests
        t0 = time.perf_counter()
        ts = [srv.submit(q[0], q[1], w.lam, w.max_iter) for q in qs * 2]
        for t in ts:
            srv.poll(t, timeout_us=60_000_000, out=out)
        capacity = len(ts) / (time.perf_counter() - t0)
        rates = []
        for frac in (0.1, 0.5, 0.9, 1.2):
            rate = frac * capacity
            n_rate = max(n_requests // 10, 16) if frac < 0.5 else n_requests
            arrivals = np.cumsum(rng.exponential(1.0 / rate, n_rate))
            sub_t, done_t, tickets, qidx = {}, {}, [], {}
            lock = th.Lock()
            finished = th.Event()

            def submitter():
                start = time.perf_counter()
                for k, a in enumerate(arrivals):
                    delay = start + a - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    q = qs[k % len(qs)]
                    tk = srv.submit(q[0], q[1], w.lam, w.max_iter)
                    with lock:
                        sub_t[tk] = time.perf_counter()
                        tickets.append(tk)
                        qidx[tk] = k % len(qs)
                finished.set()

            th_sub = th.Thread(target=submitter)
            t_start = time.perf_counter()
            th_sub.start()
            pending = []
            taken = 0
            buf = np.empty(c.N, np.float64)
            while True:
                with lock:
                    pending.extend(tickets[taken:])
                    taken = len(tickets)
                    all_in = finished.is_set() and taken == len(tickets)
                if all_in and not pending:
                    break
                for tk in list(pending):
                    try:
                        srv.poll(tk, timeout_us=0, out=buf)
                    except wmd.WMDError as e:
                        if e.status == wmd.WMD_ERR_NOT_READY:
                            continue
                        raise
                    done_t[tk] = time.perf_counter()
                    pending.remove(tk)
                    with lock:
                        qk = qidx[tk]
                    if qk < n_checked and qk not in served:
                        served[qk] = buf.copy()
                time.sleep(0.0002)
            th_sub.join()
            lat = np.array([done_t[t] - sub_t[t] for t in done_t]) * 1e3
            rates.append({"offered_qps": rate, "fraction_of_capacity": frac,
                          "achieved_qps": len(done_t) / (max(done_t.values()) - t_start),
                          "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99)),
                          "requests": len(lat)})
        stats = srv.stats()
    finally:
        srv.close()
        corpus.close()
    err = None
    if served:
        # after the timed rates: the oracle workers load the host cores
        from oracle.pool import OraclePool, sample_documents
        docs = sample_documents(c.doc_ptr, 200)
        worst, worst_q, t0 = 0.0, -1, time.perf_counter()
        with OraclePool(w.cfg) as pool:
            futs = {k: pool.submit(qs[k][0], qs[k][1], w.lam, w.max_iter, docs) for k in served}
            for k, f in futs.items():
                ref, _ = f.result(timeout=3600)
                e = error_vs_oracle(served[k][docs], ref, wmd_prec_fp32())
                if e["max_rel"] > worst:
                    worst, worst_q = e["max_rel"], k
        err = {"max_rel": worst, "worst_request_query": worst_q, "requests": len(served),
               "documents": int(docs.size), "tolerance": 1e-5,
               "v_r": sorted(int(len(qs[k][0])) for k in served),
               "oracle_wall_s": time.perf_counter() - t0,
               "sample": f"the first served result of {len(served)} distinct queries, each on "
                         f"{docs.size} seeded documents (20 longest and 20 shortest included)"}
    return {"workload": (f"serving against {w.name} corpus: V={w.V} N={w.N} docs of "
                         f"{w.doc_lo}-{w.doc_hi} words, queries v_r U[5,200], lambda={w.lam:g}, "
                         f"max_iter={w.max_iter}, Poisson arrivals, {n_requests} requests per rate "
                         f"({max(n_requests // 10, 16)} at 0.1x)"),
            "error_vs_oracle": err,
            "one_at_a_time_qps": single_qps, "capacity_qps": capacity,
            "capacity_wmds_per_s": capacity * c.N, "one_at_a_time_wmds_per_s": single_qps * c.N,
            "rates": rates, "server": {"max_batch": 32, "slots": 3, "batches": stats["batches"],
                                       "max_batch_seen": stats["max_batch_seen"]}}


_ALU_PEAK = {}


def alu_peak_tflops(device, sm_max_mhz):
    """FP32 FMA peak of the fused loop's roofline, measured on the device by
    ``wmd_measure_fp32_peak`` (the faster of packed FFMA2 and scalar FFMA).
    Returns (TFLOP/s, details); the details also carry the figure derived
    from the SM count x 128 FP32 lanes x 2 flop x the maximum SM clock."""
    import torch
    from paper_2005_06727_gb300 import wmd
    idx = torch.device(device).index or 0
    if idx not in _ALU_PEAK:
        sms = torch.cuda.get_device_properties(idx).multi_processor_count
        measured = {"ffma2": wmd.measure_fp32_peak(idx, True),
                    "ffma": wmd.measure_fp32_peak(idx, False)}
        _ALU_PEAK[idx] = (max(measured.values()),
                          {"measured_tflops": measured, "sms": sms,
                           "derived_tflops": sms * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12})
    return _ALU_PEAK[idx]


def bench_large(wmd, device, steps=5):
    """The large workload (V = N = 100,000, 20-200 Zipf words per document,
    about 11 M nonzeros, v_r = 64): one query per step (cdist + fused loop,
    CUDA events on the launching stream, L2 flushed between steps) with K
    stored in float32 and in bfloat16 (float32 arithmetic), each compared with
    the FP64 oracle on the same seeded document sample."""
    import torch
    w = synth.LARGE
    vecs, c, qs = synth.make_workload(w)
    q_ids, q_w = qs[0]
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    corpus = wmd.Corpus.from_synth(vecs, c, device=device)
    peaks, _ = measured_peaks()
    alu, _ = alu_peak_tflops(dev, peaks.get("sm_max_mhz", 2070.0))
    flops = 4.0 * len(q_ids) * c.nnz * (w.max_iter + 1)
    rec, results = {}, {}
    for name, prec in (("fp32", wmd.PREC_FP32), ("bf16_k", wmd.PREC_BF16_K)):
        variant = corpus.autotune(q_ids, q_w, w.lam, w.max_iter, prec)
        dq = wmd.DeviceQuery(corpus, q_ids, q_w, prec)
        ev = []
        for k in range(steps + 2):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            corpus.build_kernel_matrix(dq.ids, dq.w, dq.v_r, w.lam, prec, dq.ws, dq.ws_bytes, stream)
            e[1].record(stream)
            corpus.sinkhorn_loop(dq.v_r, w.max_iter, prec, dq.ws, dq.ws_bytes, dq.out, stream)
            e[2].record(stream)
            if k >= 2:
                ev.append(e)
        torch.cuda.synchronize()
        cd = statistics.mean(a.elapsed_time(b) for a, b, _ in ev)
        lp = statistics.mean(b.elapsed_time(cc) for _, b, cc in ev)
        st = statistics.mean(a.elapsed_time(cc) for a, _, cc in ev)
        results[name] = dq.out[: c.N].cpu().numpy()
        rec[name] = {"ms_per_step": st, "cdist_ms": cd, "loop_ms": lp, "value": c.N / (st * 1e-3),
                     "unit": UNIT, "loop_tflops": flops / (lp * 1e-3) / 1e12,
                     "loop_alu_frac": flops / (lp * 1e-3) / 1e12 / alu, "loop_variant": variant}
    corpus.close()
    docs = oracle_docs(c)
    from oracle.pool import OraclePool
    t0 = time.perf_counter()
    with OraclePool(w.cfg) as pool:
        chunks = [ch for ch in np.array_split(docs, pool.workers) if ch.size]
        futs = [pool.submit(q_ids, q_w, w.lam, w.max_iter, ch) for ch in chunks]
        ref = np.concatenate([f.result(timeout=3600)[0] for f in futs])
    rec["fp32"]["error_vs_oracle"] = error_vs_oracle(results["fp32"][docs], ref, wmd.PREC_FP32)
    rec["bf16_k"]["error_vs_oracle"] = error_vs_oracle(results["bf16_k"][docs], ref, wmd.PREC_BF16_K)
    rec["workload"] = (f"{w.name}: V={w.V} d={w.d} N={w.N} docs of {w.doc_lo}-{w.doc_hi} Zipf(1.1) "
                       f"words ({c.nnz} nonzeros), v_r={len(q_ids)}, lambda={w.lam:g}, "
                       f"max_iter={w.max_iter}")
    rec["oracle_sample"] = (f"{docs.size} of {c.N} documents (seeded, 20 longest and 20 shortest "
                            f"included), oracle in {time.perf_counter() - t0:.1f} s on spawned workers")
    rec["l2"] = "flushed between steps (512 MiB write)"
    return rec


def bench_paper_exact(wmd, device, steps=20):
    """The paper's own corpus shape (5000 documents, about 173k nonzeros, 34.5
    words per document; queries of 19 and 43 words): per query cdist + fused
    loop (CUDA events on the launching stream, L2 flushed between steps), the
    loop against the measured FP32 FMA rate, and every document against the
    FP64 oracle."""
    import torch
    w = synth.PAPER_EXACT
    vecs = synth.make_vecs(w.V, w.d, synth.embed_seed(w.cfg))
    c = synth.make_corpus(w.V, w.N, w.doc_lo, w.doc_hi, synth.corpus_seed(w.cfg))
    qs = synth.paper_exact_queries()
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    corpus = wmd.Corpus.from_synth(vecs, c, device=device)
    peaks, _ = measured_peaks()
    alu, _ = alu_peak_tflops(dev, peaks.get("sm_max_mhz", 2070.0))
    rows, outs = [], []
    for q_ids, q_w in qs:
        variant = corpus.autotune(q_ids, q_w, w.lam, w.max_iter)
        dq = wmd.DeviceQuery(corpus, q_ids, q_w)
        ev = []
        for k in range(steps + 3):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            e[0].record(stream)
            corpus.query_device(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter, wmd.PREC_FP32, dq.ws,
                                dq.ws_bytes, dq.out, stream)
            e[1].record(stream)
            if k >= 3:
                ev.append(e)
        lps = []
        for k in range(steps + 3):
            flush.zero_()
            corpus.build_kernel_matrix(dq.ids, dq.w, dq.v_r, w.lam, wmd.PREC_FP32, dq.ws,
                                       dq.ws_bytes, stream)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            corpus.sinkhorn_loop(dq.v_r, w.max_iter, wmd.PREC_FP32, dq.ws, dq.ws_bytes, dq.out,
                                 stream)
            b.record(stream)
            if k >= 3:
                lps.append((a, b))
        torch.cuda.synchronize()
        st = statistics.mean(a.elapsed_time(b) for a, b in ev)
        lp = statistics.mean(a.elapsed_time(b) for a, b in lps)
        flops = 4.0 * len(q_ids) * c.nnz * (w.max_iter + 1)
        outs.append(dq.out[: c.N].cpu().numpy())
        rows.append({"v_r": len(q_ids), "ms_per_step": st, "value": c.N / (st * 1e-3), "unit": UNIT,
                     "loop_ms": lp, "loop_tflops": flops / (lp * 1e-3) / 1e12,
                     "loop_alu_frac": flops / (lp * 1e-3) / 1e12 / alu, "loop_variant": variant,
                     "loop_partition": corpus.loop_partition(len(q_ids), variant)})
    corpus.close()
    docs = np.arange(c.N)
    from oracle.pool import OraclePool
    t0 = time.perf_counter()
    with OraclePool(w.cfg) as pool:
        chunks = [ch for ch in np.array_split(docs, pool.workers) if ch.size]
        for row, (q_ids, q_w), got in zip(rows, qs, outs):
            futs = [pool.submit(q_ids, q_w, w.lam, w.max_iter, ch) for ch in chunks]
            ref = np.concatenate([f.result(timeout=3600)[0] for f in futs])
            row["error_vs_oracle"] = error_vs_oracle(got, ref, wmd.PREC_FP32)
    return {"workload": (f"{w.name}: V={w.V} d={w.d} N={w.N} docs of {w.doc_lo}-{w.doc_hi} "
                         f"Zipf(1.1) words ({c.nnz} nonzeros, the paper's 173,087), queries of "
                         f"19 and 43 words, lambda={w.lam:g}, max_iter={w.max_iter}"),
            "rows": rows, "oracle": f"all {c.N} documents, {time.perf_counter() - t0:.1f} s on "
                                    f"spawned workers", "l2": "flushed between steps (512 MiB write)"}


# ------------------------------------------------------------------ ours
def bench_converge(wmd, corpus, dq, w, prec, stream, flush, reps=10):
    """Algorithm 1's "while x changes" (wmd_query_device_tol) against the
    fixed-count loop at the same cap, on the bench's corpus and query: time per
    query (CUDA events, L2 flushed before each), WMDs/s, and how many bodies
    the documents ran."""
    import torch
    N = corpus.N
    iters = torch.empty(max(N, 1), dtype=torch.int32, device=dq.out.device)
    rows = []
    for T, tol in [(15, 1e-3), (100, 1e-2), (100, 1e-3)]:
        def fixed():
            corpus.query_device(dq.ids, dq.w, dq.v_r, w.lam, T, prec, dq.ws, dq.ws_bytes, dq.out,
                                stream)

        def conv():
            corpus.query_device_tol(dq.ids, dq.w, dq.v_r, w.lam, T, tol, prec, dq.ws, dq.ws_bytes,
                                    dq.out, iters, stream)

        times = {}
        for name, fn in (("fixed", fixed), ("until_converged", conv)):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b))
            times[name] = statistics.mean(ts)
        it = iters[:N].cpu().numpy()
        rows.append({"max_iter": T, "tol": tol,
                     "fixed_ms": times["fixed"], "until_converged_ms": times["until_converged"],
                     "fixed_wmds_per_s": N / (times["fixed"] * 1e-3),
                     "until_converged_wmds_per_s": N / (times["until_converged"] * 1e-3),
                     "speedup": times["fixed"] / times["until_converged"],
                     "mean_bodies": float(it.mean()), "max_bodies": int(it.max()),
                     "stopped_before_cap": float(np.mean(it < T))})
    return {"what": "per query: cdist + fused loop, stopping each document once "
                    "max_i |x' - x| / x <= tol (capped at max_iter) vs max_iter bodies for all",
            "rows": rows}


def bench_topk(wmd, dq, N, stream, reps=20, corpus=None, w=None, prec=0, flush=None):
    """k nearest documents: wmd_topk on the bench query's WMD[N] (paper shape)
    and on a WMD-like vector of the serving corpus's size (N = 200000), CUDA
    events around each call (inputs in L2: one selection follows the loop
    that wrote them)."""
    import torch
    rows = []
    big = torch.from_numpy(1.2 + 0.3 * np.random.default_rng(0).random(200_000)).to(dq.out.device)
    for name, src, n in (("paper-shaped WMD output", dq.out, N), ("N=200000 WMD-like values", big, 200_000)):
        for k in (10, 100, 1024):
            idx = torch.empty(k, dtype=torch.int64, device=src.device)
            val = torch.empty(k, dtype=torch.float64, device=src.device)
            for _ in range(3):
                wmd.topk(src, n, k, idx, val, stream)
            ts = []
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                wmd.topk(src, n, k, idx, val, stream)
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b) * 1e3)
            rows.append({"input": name, "N": n, "k": k, "us": statistics.mean(ts)})
    out = {"what": "one-CTA radix select of the k smallest WMD values (ties to the lower id): "
                   "keys in registers, 10-bit digits of key - min for N <= 16384 and k <= 256, else "
                   "8-bit digits over shared-memory or streamed keys",
           "rows": rows}
    if corpus is not None:
        # the retrieval call against the plain query, L2 flushed before each:
        # what the selection adds to a query when it runs as the loop's
        # programmatic dependent
        def per_call(fn):
            for _ in range(3):
                fn()
            ts = []
            for _ in range(reps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ts.append(a.elapsed_time(b) * 1e3)
            return statistics.median(ts)
        plain = per_call(lambda: corpus.query_device(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter, prec,
                                                     dq.ws, dq.ws_bytes, dq.out, stream))
        added = []
        for k in (10, 100):
            idx = torch.empty(k, dtype=torch.int64, device=dq.out.device)
            val = torch.empty(k, dtype=torch.float64, device=dq.out.device)
            t = per_call(lambda: corpus.query_device_topk(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter,
                                                          prec, dq.ws, dq.ws_bytes, dq.out, k, idx,
                                                          val, stream))
            added.append({"k": k, "query_topk_us": t, "added_us": t - plain})
        out["query_device_us"] = plain
        out["query_device_topk"] = added
    return out


def bench_dense(wmd, corpus, dq, w, stream, flush, reps=5):
    """Algorithm 1 in its dense form on the same GPU (wmd_query_dense: cuBLAS
    SGEMMs for K^T u and K v over the active vocabulary, elementwise c ./ S)
    against the sparse fused path, same query and max_iter, L2 flushed before
    each call: the measured version of the paper's dense-versus-sparse
    argument (Sec. 3, Table 1)."""
    import torch
    nbytes = corpus.dense_workspace_bytes(dq.v_r)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dq.out.device)
    corpus.dense_load_c(ws, nbytes, stream)
    out = torch.empty_like(dq.out)

    def run(fn):
        for _ in range(2):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.mean(ts)

    dense_ms = run(lambda: corpus.query_dense(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter, ws, nbytes,
                                              out, stream))
    sparse_ms = run(lambda: corpus.query_device(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter,
                                                wmd.PREC_FP32, dq.ws, dq.ws_bytes, dq.out, stream))
    a = out[: corpus.N].cpu().numpy()
    b = dq.out[: corpus.N].cpu().numpy()
    rel = float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-7)))
    U, N = corpus.U, corpus.N
    return {"what": "dense Algorithm 1 (S = K^T u over all U x N positions, v = c ./ S, x = K v) "
                    "vs the sparse fused path, per query",
            "dense_ms": dense_ms, "sparse_ms": sparse_ms, "ratio": dense_ms / sparse_ms,
            "dense_wmds_per_s": N / (dense_ms * 1e-3), "workspace_bytes": nbytes,
            "dense_positions": U * N, "nonzeros": corpus.nnz,
            "max_rel_diff_dense_vs_sparse": rel}


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)

    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd

    prec = wmd.PREC_BF16_K if args.prec == "bf16" else wmd.PREC_FP32
    vecs, c, qs = synth.make_workload(w)
    q_ids, q_w = qs[0]
    corpus = wmd.Corpus.from_synth(vecs, c, device=local_rank)
    # setup (untimed): the autotuner picks the fused-loop tile variant (a
    # profiler distorts its timings: pin the variant with --loop-variant there)
    if args.loop_variant >= 0:
        corpus.set_loop_variant(len(q_ids), args.loop_variant, prec)
        corpus.set_loop_partition(len(q_ids), args.loop_variant, args.loop_partition)
        loop_variant = args.loop_variant
    else:
        loop_variant = corpus.autotune(q_ids, q_w, w.lam, w.max_iter, prec)
    loop_partition = corpus.loop_partition(len(q_ids), loop_variant)
    dq = wmd.DeviceQuery(corpus, q_ids, q_w, prec)
    v_r = dq.v_r
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        corpus.build_kernel_matrix(dq.ids, dq.w, v_r, w.lam, prec, dq.ws, dq.ws_bytes, stream)
        corpus.sinkhorn_loop(v_r, w.max_iter, prec, dq.ws, dq.ws_bytes, dq.out, stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    # timed steps: the two kernels back to back, as a caller runs them (the
    # loop kernel is a programmatic dependent of the cdist kernel and may
    # start its CTAs while that kernel finishes; an event between the two
    # would serialise them)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                       # L2 flush (untimed, between steps)
        e0, e2 = ev[k]
        e0.record(stream)
        step()
        e2.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    value, step_ms_max = replica_throughput(step_ms, c.N, world)

    # per-kernel times (the roofline of each kernel) from separate steps with
    # an event between the two kernels
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        e0, e1, e2 = kev[k]
        e0.record(stream)
        corpus.build_kernel_matrix(dq.ids, dq.w, v_r, w.lam, prec, dq.ws, dq.ws_bytes, stream)
        e1.record(stream)
        corpus.sinkhorn_loop(v_r, w.max_iter, prec, dq.ws, dq.ws_bytes, dq.out, stream)
        e2.record(stream)
    torch.cuda.synchronize()
    cdist_ms = sum(a.elapsed_time(b) for a, b, _ in kev) / args.steps
    loop_ms = sum(b.elapsed_time(cc) for _, b, cc in kev) / args.steps

    # end to end through the public host API: pinned query in, WMD[N] out
    h_ids = torch.from_numpy(np.ascontiguousarray(q_ids)).pin_memory()
    h_w = torch.from_numpy(np.ascontiguousarray(q_w)).pin_memory()
    h_out = torch.empty(c.N, dtype=torch.float64).pin_memory()
    ids_np, w_np, out_np = h_ids.numpy(), h_w.numpy(), h_out.numpy()
    for _ in range(2):
        corpus.query(ids_np, w_np, w.lam, w.max_iter, prec, out=out_np)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        corpus.query(ids_np, w_np, w.lam, w.max_iter, prec, out=out_np)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = statistics.mean(e2e_t) * 1e3
    e2e_value, _ = replica_throughput(e2e_ms, c.N, world)
    dev_out = dq.out[: c.N].cpu().numpy()
    assert np.array_equal(dev_out, out_np), "device and host paths disagree"

    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    U, ldv = corpus.U, w.d
    VR = 8
    while VR < v_r:
        VR *= 2
    kelem = 2 if prec == wmd.PREC_BF16_K else 4
    # fp16 hi + lo rows of the active vocabulary, K, norms and row scales, the query rows
    cdist_bytes = U * ldv * 4 + U * VR * kelem + U * 8 + v_r * ldv * 4
    loop_flops = 4.0 * v_r * c.nnz * (w.max_iter + 1)
    alu_tf, alu_info = alu_peak_tflops(dev, peaks.get("sm_max_mhz", 2070.0))
    alu_peak = alu_tf * 1e12
    kernels = {
        "cdist_k": {"ms": cdist_ms, "bound": "hbm", "bytes": cdist_bytes,
                    "achieved_gbs": cdist_bytes / (cdist_ms * 1e-3) / 1e9},
        "sinkhorn_fused": {"ms": loop_ms, "bound": "alu", "flops": loop_flops,
                           "achieved_tflops": loop_flops / (loop_ms * 1e-3) / 1e12,
                           "k_gather_bytes": c.nnz * VR * kelem},
    }
    if cdist_ms >= loop_ms:
        ach = cdist_bytes / (cdist_ms * 1e-3) / 1e9
        roof = {"kernel": "cdist_k", "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                "traffic": recorded_traffic("cdist_k", w.name),
                "peak_source": f"{peak_kind} hbm_gbs (copy, burst)"}
    else:
        ach = loop_flops / (loop_ms * 1e-3) / 1e12
        pk = alu_peak / 1e12
        roof = {"kernel": "sinkhorn_fused", "bound": "alu", "achieved": ach, "peak": pk,
                "unit": "TFLOP/s", "frac": ach / pk, "traffic": recorded_traffic("sinkhorn_fused", w.name, loop_variant, loop_partition),
                "peak_source": "measured FP32 FMA rate of this GPU (wmd_measure_fp32_peak, faster of "
                               "FFMA2 and FFMA)", "peak_detail": alu_info}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": step_ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == wmd.PREC_FP32 else "bf16-K/f32",
        "data": "synthetic (seeded Zipf(1.1) corpus, N(0,1/d) embeddings)",
        "config": {"workload": workload_name(w), "V": w.V, "d": w.d, "N": w.N, "v_r": v_r,
                   "lambda": w.lam, "max_iter": w.max_iter, "nnz": c.nnz, "active_words": U,
                   "loop_variant": loop_variant, "loop_partition": loop_partition,
                   "cdist_kernel": corpus.cdist_kernel,
                   "l2": "flushed between steps (512 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(v_r * 8),
                "d2h_bytes_per_step": int(c.N * 8), "ms_per_step": e2e_ms,
                "path": "wmd_query: the kernels read the query from mapped pinned memory and write WMD[N] into the pinned output"},
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    out["effective_hbm"] = effective_hbm(w, c, v_r, loop_ms, step_ms, peaks["hbm_gbs"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"], docs, ref = cpu_baseline(w, vecs, c, q_ids, q_w)
        out["error_vs_oracle"] = error_vs_oracle(out_np if docs is None else out_np[docs], ref, prec)
    legs = set(args.legs.split(",")) if args.legs else set()
    # the extra legs run on single-GPU runs only: under torchrun the other
    # ranks are done after the timed region, and the scaling runs need only it
    if rank == 0 and world == 1 and not args.no_systems:
        if "converge" in legs:
            out["converge"] = bench_converge(wmd, corpus, dq, w, prec, stream, flush)
        if "topk" in legs:
            out["topk"] = bench_topk(wmd, dq, c.N, stream, corpus=corpus, w=w, prec=prec,
                                     flush=flush)
        if "dense" in legs and prec == wmd.PREC_FP32:
            out["dense"] = bench_dense(wmd, corpus, dq, w, stream, flush)
        if "large" in legs:
            out["large"] = bench_large(wmd, local_rank)
        if "paper_exact" in legs:
            out["paper_exact"] = bench_paper_exact(wmd, local_rank)
        if "batched" in legs:
            out["batched"] = bench_batched(wmd, local_rank, with_oracle=not args.no_cpu_baseline)
        if "serving" in legs:
            out["serving"] = bench_serving(wmd, local_rank, args.serve_requests,
                                           workload=args.serving_workload)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # last, after every GPU leg: its worker processes load the host, and the
        # one-at-a-time leg above is host-bound (it measured 0.34 instead of
        # 0.19 s when this ran before it)
        try:
            out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(w, c, oracle_docs(c))
        except Exception as e:  # a host without spawn support: report, do not fail the bench
            out["cpu_baseline_all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out))
    corpus.close()
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args, w):
    """The document-sharded path: rank r holds the r-th nnz-balanced document
    range of the corpus (wmd_corpus_load_shard); a step is one query on every
    shard (cdist + fused loop) followed by the exchange step, an all_gather of
    the WMD slices, so that every rank ends with all N values.  Total work is
    fixed as ranks are added (strong scaling)."""
    import torch
    import torch.distributed as dist
    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import shard, wmd
    prec = wmd.PREC_BF16_K if args.prec == "bf16" else wmd.PREC_FP32
    vecs, c, qs = synth.make_workload(w)
    q_ids, q_w = qs[0]
    bounds = shard.plan(c.row_ptr, c.doc_idx, c.V, c.N, world)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    corpus = shard.load_shard(vecs, c.row_ptr, c.doc_idx, c.val, c.N, lo, hi, device=local_rank)
    variant = corpus.autotune(q_ids, q_w, w.lam, w.max_iter, prec) if corpus.N else 0
    dq = wmd.DeviceQuery(corpus, q_ids, q_w, prec)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    counts = np.diff(bounds)

    def step():
        if corpus.N:
            corpus.build_kernel_matrix(dq.ids, dq.w, dq.v_r, w.lam, prec, dq.ws, dq.ws_bytes, stream)
            corpus.sinkhorn_loop(dq.v_r, w.max_iter, prec, dq.ws, dq.ws_bytes, dq.out, stream)
        local = dq.out[: corpus.N]
        return shard.gather_slices(local, counts) if world > 1 else local

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    times = []
    clocks = ClockSampler(local_rank)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        full = step()
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = statistics.mean(a.elapsed_time(b) for a, b in times)
    t = torch.tensor([step_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    step_max = float(t.item())
    # end to end: the same step with the result copied to the host
    e2e = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        host = step().cpu().numpy()
        e2e.append(time.perf_counter() - t0)
    e2e_ms = statistics.mean(e2e) * 1e3
    te = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    assert host.shape == (c.N,)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": c.N / (step_max * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": step_max,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if prec == wmd.PREC_FP32 else "bf16-K/f32",
            "data": "synthetic (seeded Zipf(1.1) corpus, N(0,1/d) embeddings)",
            "gpu_launches": 2 * args.steps,
            "config": {"workload": workload_name(w), "V": w.V, "d": w.d, "N": w.N,
                       "v_r": dq.v_r, "lambda": w.lam, "max_iter": w.max_iter,
                       "parallelism": f"documents sharded x{world} (nnz-balanced), all_gather of "
                                      "the WMD slices every step",
                       "shard_docs": [int(x) for x in counts], "loop_variant": variant,
                       "l2": "flushed between steps (512 MiB write)"},
            "e2e": {"value": c.N / (float(te.item()) * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(c.N * 8),
                    "ms_per_step": float(te.item()),
                    "path": "device query on every shard, all_gather, WMD[N] copied to the host"},
            "clocks": clk}))
    corpus.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
    elif args.shard_docs:
        run_sharded(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
