"""The dense Algorithm 1 comparator (wmd_query_dense) against the FP64 oracle.

The dense form computes K^T u at every (word, document) position and scales
the dense c with it (Algorithm 1 as written, the form Sec. 3 argues against);
it must give the same WMD as the sparse path: within 1e-5 relative of the
oracle (whose dense and sparse forms are pinned equal), NaN on empty
documents, and within the same tolerance of the GPU's sparse result.
"""
import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module")
def wmd():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd as w
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return w


def _parity(got, want, rtol, what):
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan), f"{what}: NaN pattern differs"
    rel = np.abs(got[~nan] - want[~nan]) / np.maximum(np.abs(want[~nan]), 1e-7)
    assert rel.size == 0 or rel.max() <= rtol, f"{what}: max rel err {rel.max():.3e}"


class Dense:
    def __init__(self, wmd, corpus, v_r):
        import torch
        self.corpus = corpus
        self.bytes = corpus.dense_workspace_bytes(v_r)
        self.ws = torch.empty(self.bytes, dtype=torch.uint8, device="cuda")
        corpus.dense_load_c(self.ws, self.bytes)
        self.out = torch.empty(max(corpus.N, 1), dtype=torch.float64, device="cuda")

    def run(self, wmd, q_ids, q_w, lam, T):
        import torch
        ids, w = wmd.compact_query(q_ids, q_w, self.corpus.V)
        d_ids = torch.from_numpy(ids).cuda()
        d_w = torch.from_numpy(w).cuda()
        self.corpus.query_dense(d_ids, d_w, ids.size, lam, T, self.ws, self.bytes, self.out)
        torch.cuda.synchronize()
        return self.out.cpu().numpy()[: self.corpus.N]


def _oracle(vecs, c, q_ids, q_w, lam, T):
    return orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N, vecs, lam, T)


def test_tiny_workload_dense(wmd):
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    d = Dense(wmd, corpus, len(q_ids))
    for T in (0, 1, 15):
        got = d.run(wmd, q_ids, q_w, w.lam, T)
        _parity(got, _oracle(vecs, c, q_ids, q_w, w.lam, T), FP32_RTOL, f"tiny T={T}")
        _parity(got, corpus.query(q_ids, q_w, w.lam, T), FP32_RTOL, f"tiny vs sparse T={T}")


@pytest.mark.parametrize("v_r", [1, 9, 33, 100, 200])
def test_query_widths_and_empty_documents(wmd, v_r):
    V = 3000
    vecs = synth.make_vecs(V, 300, 70 + v_r)
    c0 = synth.make_corpus(V, 40, 1, 60, 80 + v_r)
    docs = [(c0.doc_words[c0.doc_ptr[j]:c0.doc_ptr[j + 1]], c0.doc_vals[c0.doc_ptr[j]:c0.doc_ptr[j + 1]])
            for j in range(c0.N)]
    docs.insert(5, (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    c = synth.corpus_from_docs(V, docs)
    q_ids, q_w = synth.make_query(V, v_r, 90 + v_r)
    corpus = wmd.Corpus.from_synth(vecs, c)
    d = Dense(wmd, corpus, v_r)
    for T in (0, 15):
        got = d.run(wmd, q_ids, q_w, 10.0, T)
        _parity(got, _oracle(vecs, c, q_ids, q_w, 10.0, T), FP32_RTOL, f"v_r={v_r} T={T}")


def test_paper_shaped_dense_all_documents(wmd):
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    d = Dense(wmd, corpus, len(q_ids))
    got = d.run(wmd, q_ids, q_w, w.lam, w.max_iter)
    _parity(got, _oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter), FP32_RTOL, "paper-shaped dense")
    # a second query reuses the dense c of the workspace
    q2 = synth.make_query(w.V, 17, 555)
    got2 = d.run(wmd, *q2, w.lam, w.max_iter)
    _parity(got2, corpus.query(*q2, w.lam, w.max_iter), FP32_RTOL, "paper-shaped second query")


def test_dense_workspace_too_small_is_rejected(wmd):
    import torch
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    need = corpus.dense_workspace_bytes(len(q_ids))
    assert need > 0 and corpus.dense_workspace_bytes(0) == 0
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    out = torch.empty(c.N, dtype=torch.float64, device="cuda")
    ids = torch.from_numpy(np.asarray(q_ids, np.int32)).cuda()
    wts = torch.from_numpy(np.asarray(q_w, np.float32)).cuda()
    with pytest.raises(wmd.WMDError) as e:
        corpus.query_dense(ids, wts, len(q_ids), w.lam, w.max_iter, ws, need - 256, out)
    assert e.value.status == wmd.WMD_ERR_INVALID_ARG
