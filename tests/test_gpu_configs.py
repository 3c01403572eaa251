"""Oracle parity at the sizes of the batched and the served workloads.

The batched workload (V = 100,000, d = 300, N = 20,000 documents of 20-150
Zipf words, 256 queries with v_r uniform in [5, 128]) runs as one
wmd_query_batch call; every query is compared with the FP64 oracle on a
seeded sample of 200 documents that holds the 20 longest and the 20 shortest.
The served workload (V = N = 200,000, 20-200 words per document, about 22 M
nonzeros) answers a mix of requests through wmd_serve_submit / poll,
v_r = 200 and the longest documents included (the paths where teams of
several warps re-read their chunks of K).  Tolerance: 1e-5 relative per
document (FP32), as everywhere else.

The oracle runs in spawned worker processes (oracle/pool.py) while the GPU
works; each worker rebuilds the seeded workload itself.
"""
import numpy as np
import pytest

from oracle.pool import OraclePool, sample_documents
from paper_2005_06727_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP32_RTOL = 1e-5


@pytest.fixture(scope="module")
def wmd():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd as w
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return w


def _rel(got, want):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    return np.abs(got[ok] - want[ok]) / np.maximum(np.abs(want[ok]), 1e-7)


def test_batched_workload_every_query_against_oracle(wmd):
    w = synth.BATCHED
    vecs, c, qs = synth.make_workload(w)
    assert len(qs) == 256
    docs = sample_documents(c.doc_ptr, 200)
    lens = np.diff(c.doc_ptr)
    assert lens[docs].max() == lens.max() and lens[docs].min() == lens.min()
    with OraclePool(w.cfg) as pool:
        futs = [pool.submit(q[0], q[1], w.lam, w.max_iter, docs) for q in qs]
        corpus = wmd.Corpus.from_synth(vecs, c)
        got = corpus.query_batch(qs, w.lam, w.max_iter)
        corpus.close()
        worst = 0.0
        for k, f in enumerate(futs):
            want, _ = f.result(timeout=1800)
            rel = _rel(got[k][docs], want)
            assert rel.max() <= FP32_RTOL, f"query {k} (v_r={len(qs[k][0])}): {rel.max():.3e}"
            worst = max(worst, float(rel.max()))
    print(f"batched workload: 256 queries x {docs.size} documents, max rel err {worst:.2e}")


def test_serving_workload_requests_against_oracle(wmd):
    w = synth.SERVING
    widths = [200, 5, 128, 129, 64, 65, 33, 17, 9, 8, 150, 100, 77, 31, 190, 42, 256 - 1, 12]
    qs = [synth.make_query(w.V, vr, 70_000 + i) for i, vr in enumerate(widths)]
    with OraclePool(w.cfg) as pool:
        vecs = synth.make_vecs(w.V, w.d, synth.embed_seed(w.cfg))
        c = synth.make_corpus(w.V, w.N, w.doc_lo, w.doc_hi, synth.corpus_seed(w.cfg))
        docs = sample_documents(c.doc_ptr, 200)
        futs = [pool.submit(q[0], q[1], w.lam, w.max_iter, docs) for q in qs]
        corpus = wmd.Corpus.from_synth(vecs, c)
        srv = wmd.Server(corpus, max_batch=8, slots=3, mem_budget=24 << 30)
        try:
            tickets = [srv.submit(q[0], q[1], w.lam, w.max_iter) for q in qs]
            served = [srv.poll(t, timeout_us=600_000_000) for t in tickets]
            stats = srv.stats()
        finally:
            srv.close()
        assert stats["completed"] == len(qs) and stats["batches"] >= 2
        # a request's result does not depend on the mix it was served in
        for k in (0, 1, 14):
            np.testing.assert_array_equal(corpus.query(qs[k][0], qs[k][1], w.lam, w.max_iter),
                                          served[k])
        corpus.close()
        worst = 0.0
        for k, f in enumerate(futs):
            want, _ = f.result(timeout=1800)
            rel = _rel(served[k][docs], want)
            assert rel.max() <= FP32_RTOL, f"request {k} (v_r={widths[k]}): {rel.max():.3e}"
            worst = max(worst, float(rel.max()))
    print(f"served workload: {len(qs)} requests x {docs.size} documents, max rel err {worst:.2e}")
