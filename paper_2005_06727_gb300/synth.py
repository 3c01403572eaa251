"""Seeded synthetic inputs shaped like the paper's WMD workload.

The paper (Sec. 3, "Dataset") measures on 100,000 fastText crawl-300d words and
the first 5000 dbpedia documents.  Those files are not available here, so this
module draws stand-ins of the same shape:

* ``vecs``: V x d embeddings, entries N(0, 1/d), drawn in float64 and rounded to
  float32 (the paper's table is a dense V x w matrix, Sec. 3).
* documents: word ids drawn i.i.d. from Zipf(s=1.1) over a frequency-ordered
  vocabulary (rank k -> id k-1) until the document holds ``n_j`` distinct ids,
  ``n_j ~ U{lo..hi}``; weights are the drawn counts divided by their total, in
  float64, then rounded to float32 (the columns of ``c`` "sum to 1", Sec. 3).
* ``c`` is returned in the paper's layout: a V x N CSR matrix with rows = words.
* queries are drawn like documents with ``n = v_r`` distinct words.

This module holds no arithmetic of the method itself (no distances, kernels or
scaling); it only produces inputs, and both the oracle tests and the CUDA path
consume them.
"""
from __future__ import annotations

import dataclasses
import numpy as np

ZIPF_S = 1.1


@dataclasses.dataclass(frozen=True)
class Workload:
    """One workload shape (vocabulary, corpus and query sizes)."""
    name: str
    V: int
    d: int
    N: int
    doc_lo: int
    doc_hi: int
    vr_lo: int
    vr_hi: int
    n_queries: int
    cfg: int          # seed namespace
    lam: float = 10.0
    max_iter: int = 15


# The five workloads of the hot path (sizes from the paper's Sec. 3 shape,
# scaled up for the large / batched / served cases).
TINY = Workload("tiny V=2000 N=100 v_r=20", 2000, 300, 100, 10, 40, 20, 20, 1, 1)
PAPER = Workload("paper-shaped V=100000 N=5000 v_r=30", 100_000, 300, 5000, 20, 150, 30, 30, 1, 2)
LARGE = Workload("large V=100000 N=100000 v_r=64", 100_000, 300, 100_000, 20, 200, 64, 64, 1, 3)
BATCHED = Workload("batched V=100000 N=20000 256 queries v_r U[5,128]", 100_000, 300, 20_000, 20, 150, 5, 128, 256, 4)
SERVING = Workload("serving V=200000 N=200000 v_r U[5,200]", 200_000, 300, 200_000, 20, 200, 5, 200, 2000, 5)

# The paper's own corpus shape (Sec. 3: the first 5000 dbpedia documents,
# 173,087 nonzeros, 34.6 distinct words per document on average; its queries
# have 19 and 43 words): documents of U{10..59} words, queries of 19 and 43.
PAPER_EXACT = Workload("paper-exact V=100000 N=5000 v_r 19 and 43", 100_000, 300, 5000, 10, 59, 19, 43,
                       2, 6)
PAPER_EXACT_VR = (19, 43)

WORKLOADS = {w.cfg: w for w in (TINY, PAPER, LARGE, BATCHED, SERVING, PAPER_EXACT)}


def paper_exact_queries() -> list[tuple[np.ndarray, np.ndarray]]:
    """The two queries of the paper-exact workload, 19 and 43 words."""
    return [make_query(PAPER_EXACT.V, vr, query_seed(PAPER_EXACT.cfg, q))
            for q, vr in enumerate(PAPER_EXACT_VR)]


def corpus_seed(cfg: int) -> int:
    return 1000 + cfg


def query_seed(cfg: int, q: int) -> int:
    return 2000 + cfg * 1000 + q


def embed_seed(cfg: int) -> int:
    return 7 + cfg


def zipf_cdf(V: int, s: float = ZIPF_S) -> np.ndarray:
    """Cumulative distribution of P(rank k) proportional to k^-s, k = 1..V."""
    p = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(p)
    cdf /= cdf[-1]
    return cdf


def _draw_bag(rng: np.random.Generator, cdf: np.ndarray, n: int,
              perm: np.ndarray | None) -> tuple[np.ndarray, np.ndarray]:
    """Draw Zipf tokens until ``n`` distinct ids were seen.

    Returns sorted unique ids (int32) and their normalised counts (float32).
    """
    V = cdf.shape[0]
    if n > V:
        raise ValueError("cannot draw more distinct words than the vocabulary holds")
    tokens = np.empty(0, dtype=np.int64)
    batch = max(4 * n, 64)
    while True:
        more = np.searchsorted(cdf, rng.random(batch), side="right")
        np.minimum(more, V - 1, out=more)
        tokens = np.concatenate([tokens, more])
        uniq, first = np.unique(tokens, return_index=True)
        if uniq.shape[0] >= n:
            cut = np.sort(first)[n - 1]          # token that brought the n-th new id
            tokens = tokens[: cut + 1]
            break
        batch *= 2
    ids, counts = np.unique(tokens, return_counts=True)
    if perm is not None:
        ids = perm[ids]
        order = np.argsort(ids, kind="stable")
        ids, counts = ids[order], counts[order]
    w = counts.astype(np.float64) / counts.sum(dtype=np.float64)
    return ids.astype(np.int32), w.astype(np.float32)


def make_vecs(V: int, d: int, seed: int) -> np.ndarray:
    """V x d float32 embeddings with entries N(0, 1/d) (drawn in float64)."""
    rng = np.random.default_rng(seed)
    out = np.empty((V, d), dtype=np.float32)
    step = 16384
    scale = 1.0 / np.sqrt(d)
    for a in range(0, V, step):
        b = min(V, a + step)
        out[a:b] = (rng.standard_normal((b - a, d)) * scale).astype(np.float32)
    return out


@dataclasses.dataclass
class Corpus:
    """The paper's ``c`` (V x N CSR, rows = words) plus its doc-major view."""
    V: int
    N: int
    row_ptr: np.ndarray      # int64 [V+1]
    doc_idx: np.ndarray      # int32 [nnz], increasing within a row
    val: np.ndarray          # float32 [nnz]
    doc_ptr: np.ndarray      # int64 [N+1]   (doc-major copy, for tests)
    doc_words: np.ndarray    # int32 [nnz]   sorted within a document
    doc_vals: np.ndarray     # float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.val.shape[0])


def corpus_from_docs(V: int, docs: list[tuple[np.ndarray, np.ndarray]]) -> Corpus:
    """Assemble the V x N CSR (rows = words) from per-document (ids, weights)."""
    N = len(docs)
    lens = np.array([len(ids) for ids, _ in docs], dtype=np.int64)
    doc_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(lens, out=doc_ptr[1:])
    if N:
        words = np.concatenate([np.asarray(ids, dtype=np.int32) for ids, _ in docs]) if doc_ptr[-1] else np.zeros(0, np.int32)
        vals = np.concatenate([np.asarray(w, dtype=np.float32) for _, w in docs]) if doc_ptr[-1] else np.zeros(0, np.float32)
    else:
        words = np.zeros(0, np.int32)
        vals = np.zeros(0, np.float32)
    docs_of = np.repeat(np.arange(N, dtype=np.int32), lens)
    order = np.argsort(words, kind="stable")           # docs already ascending
    row_counts = np.bincount(words, minlength=V).astype(np.int64)
    row_ptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(row_counts, out=row_ptr[1:])
    return Corpus(V, N, row_ptr, docs_of[order].astype(np.int32), vals[order].astype(np.float32),
                  doc_ptr, words, vals)


def make_corpus(V: int, N: int, lo: int, hi: int, seed: int,
                permute_ids: bool = False) -> Corpus:
    """N documents with U{lo..hi} distinct Zipf(1.1) words each."""
    rng = np.random.default_rng(seed)
    cdf = zipf_cdf(V)
    perm = rng.permutation(V).astype(np.int64) if permute_ids else None
    lens = rng.integers(lo, hi + 1, size=N)
    docs = [_draw_bag(rng, cdf, int(n), perm) for n in lens]
    return corpus_from_docs(V, docs)


def make_query(V: int, v_r: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """One query: sorted unique word ids (int32) and weights (float32)."""
    rng = np.random.default_rng(seed)
    return _draw_bag(rng, zipf_cdf(V), v_r, None)


def make_queries(w: Workload, count: int | None = None) -> list[tuple[np.ndarray, np.ndarray]]:
    n = w.n_queries if count is None else count
    out = []
    for q in range(n):
        if w.vr_lo == w.vr_hi:
            vr = w.vr_lo
        else:
            vr = int(np.random.default_rng(query_seed(w.cfg, q) + 500_000).integers(w.vr_lo, w.vr_hi + 1))
        out.append(make_query(w.V, vr, query_seed(w.cfg, q)))
    return out


def make_workload(w: Workload, n_queries: int | None = None):
    """(vecs, corpus, queries) for a workload, all seeded."""
    vecs = make_vecs(w.V, w.d, embed_seed(w.cfg))
    corpus = make_corpus(w.V, w.N, w.doc_lo, w.doc_hi, corpus_seed(w.cfg))
    return vecs, corpus, make_queries(w, n_queries)


def dense_r(V: int, ids: np.ndarray, w: np.ndarray) -> np.ndarray:
    """The query as the paper's dense V-vector r."""
    r = np.zeros(V, dtype=np.float64)
    r[np.asarray(ids, dtype=np.int64)] = np.asarray(w, dtype=np.float32).astype(np.float64)
    return r


def dense_c(c: Corpus) -> np.ndarray:
    """The paper's c as a dense V x N float64 matrix (tiny inputs only)."""
    out = np.zeros((c.V, c.N), dtype=np.float64)
    rows = np.repeat(np.arange(c.V), np.diff(c.row_ptr))
    out[rows, c.doc_idx] = c.val.astype(np.float64)
    return out
