"""Runs the FP64 oracle on many (query, document sample) tasks at once.

TEST INFRASTRUCTURE ONLY: imported by the test suite and by bench.py's oracle
legs (its CPU baseline and the errors it reports against the oracle).  This
module holds none of the method's arithmetic.  Every worker process rebuilds
the seeded synthetic workload itself (cheaper than shipping the arrays, and
the same bits) and calls ``sinkhorn_wmd.sinkhorn_wmd_sparse`` unchanged on the
tasks it is given.  Workers are spawned, never forked, so a pool may start
after the parent process already holds a CUDA context.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
_STATE: dict = {}


def _init(cfg: int, root: str):
    if root not in sys.path:
        sys.path.insert(0, root)
    from paper_2005_06727_gb300 import synth
    w = synth.WORKLOADS[cfg]
    _STATE["vecs"] = synth.make_vecs(w.V, w.d, synth.embed_seed(w.cfg))
    _STATE["c"] = synth.make_corpus(w.V, w.N, w.doc_lo, w.doc_hi, synth.corpus_seed(w.cfg))


def _run(task):
    from oracle import sinkhorn_wmd as orc
    q_ids, q_w, lam, max_iter, docs = task
    c = _STATE["c"]
    t0 = time.perf_counter()
    out = orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N, _STATE["vecs"],
                                  lam, max_iter, docs=docs)
    return out, time.perf_counter() - t0


class OraclePool:
    """A pool of single-threaded oracle workers for one seeded workload
    (``synth.WORKLOADS[cfg]``).  ``submit`` returns a future of
    ``(wmd[docs], seconds)``; use as a context manager."""

    def __init__(self, cfg: int, workers: int | None = None):
        self.workers = max(1, workers or os.cpu_count() or 1)
        self._saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:          # inherited by the spawned workers
            os.environ[k] = "1"
        # an executor (not multiprocessing.Pool): a worker that cannot start
        # raises BrokenProcessPool instead of being respawned for ever
        self._ex = cf.ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"),
                                          initializer=_init, initargs=(cfg, ROOT))

    def submit(self, q_ids, q_w, lam: float, max_iter: int, docs=None) -> cf.Future:
        d = None if docs is None else np.asarray(docs, dtype=np.int64)
        return self._ex.submit(_run, (np.asarray(q_ids, np.int32), np.asarray(q_w, np.float32),
                                      float(lam), int(max_iter), d))

    def close(self):
        self._ex.shutdown(wait=True, cancel_futures=True)
        for k, v in self._saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sample_documents(doc_ptr, n: int = 200, extremes: int = 20, seed: int = 0) -> np.ndarray:
    """A seeded sample of n document ids that holds the ``extremes`` longest
    and shortest documents (sorted ids)."""
    lens = np.diff(np.asarray(doc_ptr))
    N = lens.size
    order = np.argsort(lens, kind="stable")
    keep = set(order[:extremes].tolist()) | set(order[-extremes:].tolist())
    rng = np.random.default_rng(seed)
    rest = rng.permutation(N)
    for j in rest:
        if len(keep) >= min(n, N):
            break
        keep.add(int(j))
    return np.array(sorted(keep), dtype=np.int64)
