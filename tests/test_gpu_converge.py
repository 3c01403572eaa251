"""The convergence-tested loop (wmd_query_device_tol) against the FP64 oracle.

Algorithm 1 loops "while x changes"; per document j the loop stops after the
first body k with max_i |x^(k) - x^(k-1)| / x^(k-1) <= tol (capped at
max_iter).  The GPU takes that decision in float32 and the oracle in float64,
so a document whose relative change lies within rounding of tol may stop one
body apart.  The tests therefore check:

* WMD parity (1e-5 relative, as for the fixed-count path) against the oracle
  forced to the per-document body counts that the GPU reports;
* that every reported count is valid under the exact rule: the FP64 relative
  change exceeds tol before it (NaN counts as changing) and is at most tol at
  it (unless the cap was hit), up to a band of 1% of tol for float32 rounding;
* that nearly all counts equal the oracle's own.
"""
import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5
BF16_RTOL = 5e-3
BAND = 0.01


@pytest.fixture(scope="module")
def wmd():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd as w
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return w


def _run(wmd, corpus, q_ids, q_w, lam, T, tol, prec=None):
    import torch
    prec = wmd.PREC_FP32 if prec is None else prec
    ids, w = wmd.compact_query(q_ids, q_w, corpus.V)
    dev = torch.device("cuda", corpus.device)
    d_ids = torch.from_numpy(ids).to(dev)
    d_w = torch.from_numpy(w).to(dev)
    ws_bytes = corpus.workspace_bytes(ids.size, prec)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    out = torch.full((corpus.N,), -7.0, dtype=torch.float64, device=dev)
    iters = torch.full((corpus.N,), -1, dtype=torch.int32, device=dev)
    corpus.query_device_tol(d_ids, d_w, ids.size, lam, T, tol, prec, ws, ws_bytes, out, iters)
    torch.cuda.synchronize()
    return out.cpu().numpy(), iters.cpu().numpy().astype(np.int64)


def _run_fixed(wmd, corpus, q_ids, q_w, lam, T):
    import torch
    dq = wmd.DeviceQuery(corpus, q_ids, q_w)
    out = dq.run(lam, T)
    torch.cuda.synchronize()
    return out.cpu().numpy()[: corpus.N]


def _oracle(vecs, c, q_ids, q_w, lam, T, tol, iters=None, docs=None):
    return orc.sinkhorn_wmd_sparse_until_converged(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N,
                                                   vecs, lam, T, tol, iters=iters, docs=docs)


def _parity(got, want, rtol, what):
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan), f"{what}: NaN pattern differs"
    rel = np.abs(got[~nan] - want[~nan]) / np.maximum(np.abs(want[~nan]), 1e-7)
    assert rel.size == 0 or rel.max() <= rtol, f"{what}: max rel err {rel.max():.3e}"


def _check(wmd, corpus, vecs, c, q_ids, q_w, lam, T, tol, docs=None, min_exact=0.9, what=""):
    got, it = _run(wmd, corpus, q_ids, q_w, lam, T, tol)
    sel = np.arange(c.N) if docs is None else np.asarray(docs)
    assert np.all((it[sel] >= 0) & (it[sel] <= T)), f"{what}: counts out of range"
    want, forced, rho = _oracle(vecs, c, q_ids, q_w, lam, T, tol, iters=it, docs=docs)
    assert np.array_equal(forced, it[sel])
    _parity(got[sel], want, FP32_RTOL, what)
    for jj, j in enumerate(sel):
        k = it[j]
        if k == 0:
            assert T == 0
            continue
        ch = rho[:k, jj]
        assert not np.any(ch[:-1] <= tol * (1 - BAND)), f"{what}: doc {j} ran past a stop ({ch})"
        assert k == T or ch[-1] <= tol * (1 + BAND), f"{what}: doc {j} stopped early ({ch[-1]})"
    _, exact, _ = _oracle(vecs, c, q_ids, q_w, lam, T, tol, docs=docs)
    same = np.mean(exact == it[sel])
    assert same >= min_exact, f"{what}: only {same:.2%} of counts equal the exact rule's"
    return got, it


@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_tiny_workload_until_converged(wmd, tol):
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    _, it = _check(wmd, corpus, vecs, c, q_ids, q_w, w.lam, 100, tol, what=f"tiny tol={tol}")
    assert it.min() < 100 and it.max() > it.min()    # the rule stops documents at different bodies


def test_paper_shaped_sampled_documents(wmd):
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    lens = np.diff(c.doc_ptr)
    rng = np.random.default_rng(3)
    docs = np.unique(np.concatenate([rng.choice(c.N, 300, replace=False),
                                     np.argsort(lens)[-10:], np.argsort(lens)[:10]]))
    _check(wmd, corpus, vecs, c, q_ids, q_w, w.lam, 60, 1e-3, docs=docs, what="paper-shaped")


@pytest.mark.parametrize("v_r,lengths", [
    (8, [0, 3, 383, 385, 1000]),                  # one-warp teams; a chunked document
    (30, [1, 2, 0, 95, 97, 193, 700]),            # shared-memory finish; 1, 2, 4 warps
    (64, [47, 49, 97, 200, 400]),                 # register finish; teams of warps
    (200, [5, 13, 49, 300, 0]),                   # 8-warp CTAs
    (40, [3, 65, 129, 257, 0]),                   # 48-wide tile
    (90, [5, 33, 65, 129, 257, 0]),               # 96-wide tile
    (150, [5, 17, 33, 65, 129, 0]),               # 192-wide tile
])
def test_team_sizes_and_empty_documents(wmd, v_r, lengths):
    V = 4000
    vecs = synth.make_vecs(V, 300, 3)
    rng = np.random.default_rng(v_r)
    docs = []
    for n in lengths:
        ids = np.sort(rng.choice(V, n, replace=False)).astype(np.int32)
        wts = rng.random(n) + 0.05
        docs.append((ids, (wts / wts.sum()).astype(np.float32)))
    c = synth.corpus_from_docs(V, docs)
    q_ids, q_w = synth.make_query(V, v_r, 9)
    corpus = wmd.Corpus.from_synth(vecs, c)
    got, it = _check(wmd, corpus, vecs, c, q_ids, q_w, 10.0, 40, 1e-2, min_exact=0.7,
                     what=f"lengths v_r={v_r}")
    empty = np.asarray(lengths) == 0
    assert np.all(it[empty] == 40) and np.all(np.isnan(got[empty]))


def test_zero_tolerance_and_zero_iterations_match_the_fixed_loop(wmd):
    """tol = 0 stops a document only when x no longer changes at all, after
    which every further body repeats the same float32 values: the results are
    the fixed-count ones bit for bit.  max_iter = 0 runs no body."""
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    for T in (15, 1):
        got, it = _run(wmd, corpus, q_ids, q_w, w.lam, T, 0.0)
        assert np.array_equal(got, _run_fixed(wmd, corpus, q_ids, q_w, w.lam, T))
        assert np.all((it >= 1) & (it <= T))
    got, it = _run(wmd, corpus, q_ids, q_w, w.lam, 0, 1e-3)
    assert np.all(it == 0)
    assert np.array_equal(got, _run_fixed(wmd, corpus, q_ids, q_w, w.lam, 0))


def test_bf16_stored_k_until_converged(wmd):
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    got, it = _run(wmd, corpus, q_ids, q_w, w.lam, 60, 1e-2, prec=wmd.PREC_BF16_K)
    want, _, _ = _oracle(vecs, c, q_ids, q_w, w.lam, 60, 1e-2, iters=it)
    _parity(got, want, BF16_RTOL, "tiny bf16")


def test_tolerance_out_of_range_is_rejected(wmd):
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    for tol in (1.0, -1e-3, float("nan")):
        with pytest.raises(wmd.WMDError) as e:
            _run(wmd, corpus, q_ids, q_w, w.lam, 10, tol)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
