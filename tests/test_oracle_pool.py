"""The oracle's process pool (test infrastructure) returns exactly what a
direct call of the oracle returns, and the document sample holds the extremes."""
import numpy as np

from oracle import sinkhorn_wmd as orc
from oracle.pool import OraclePool, sample_documents
from paper_2005_06727_gb300 import synth


def test_pool_results_equal_direct_oracle_calls():
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    q2 = synth.make_query(w.V, 7, 99)
    docs = sample_documents(c.doc_ptr, 30)
    with OraclePool(w.cfg, workers=2) as pool:
        fa = pool.submit(qs[0][0], qs[0][1], w.lam, w.max_iter)
        fb = pool.submit(q2[0], q2[1], 3.0, 4, docs)
        a, ta = fa.result(timeout=600)
        b, tb = fb.result(timeout=600)
    assert ta > 0 and tb > 0
    np.testing.assert_array_equal(a, orc.sinkhorn_wmd_sparse(
        qs[0][0], qs[0][1], c.row_ptr, c.doc_idx, c.val, c.N, vecs, w.lam, w.max_iter))
    np.testing.assert_array_equal(b, orc.sinkhorn_wmd_sparse(
        q2[0], q2[1], c.row_ptr, c.doc_idx, c.val, c.N, vecs, 3.0, 4, docs=docs))


def test_document_sample_holds_the_extremes():
    doc_ptr = np.concatenate([[0], np.cumsum(np.arange(1, 501) % 97 + 1)])
    lens = np.diff(doc_ptr)
    s = sample_documents(doc_ptr, 100, extremes=20)
    assert s.size == 100 and np.all(np.diff(s) > 0)
    order = np.argsort(lens, kind="stable")
    assert set(order[:20]) <= set(s) and set(order[-20:]) <= set(s)
    assert np.array_equal(sample_documents(doc_ptr, 1000), np.arange(500))
