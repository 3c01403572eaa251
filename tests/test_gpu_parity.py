"""Parity of the CUDA path against the FP64 oracle (GPU only).

Tolerance: the float32 path must match the oracle within 1e-5 relative per
document (absolute floor 1e-7); the bfloat16-stored K path within 5e-3.  NaN
results (empty documents) must coincide.  Every call goes through the C ABI.
"""
import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5
BF16_RTOL = 5e-3


@pytest.fixture(scope="module")
def wmd():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd as w
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return w


def assert_parity(got, want, rtol, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape
    nan_w = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan_w), f"{what}: NaN pattern differs"
    g, w = got[~nan_w], want[~nan_w]
    rel = np.abs(g - w) / np.maximum(np.abs(w), 1e-7)
    worst = int(np.argmax(rel)) if rel.size else 0
    assert rel.size == 0 or rel.max() <= rtol, (
        f"{what}: max rel err {rel.max():.3e} at {worst}: got {g[worst]!r} want {w[worst]!r}")
    return float(rel.max()) if rel.size else 0.0


def oracle(vecs, c, q_ids, q_w, lam, T, docs=None):
    return orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N, vecs, lam, T,
                                   docs=docs)


def _docs(c):
    return [(c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]], c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]])
            for j in range(c.N)]


# ---------------------------------------------------------------- workloads
def test_tiny_workload(wmd):
    w = synth.TINY
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    want = oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter)
    got = corpus.query(q_ids, q_w, w.lam, w.max_iter)
    assert_parity(got, want, FP32_RTOL, "tiny fp32")
    got16 = corpus.query(q_ids, q_w, w.lam, w.max_iter, wmd.PREC_BF16_K)
    assert_parity(got16, want, BF16_RTOL, "tiny bf16")


def test_paper_shaped_workload_all_documents(wmd):
    """V=100000, N=5000, 20-150 words per document, v_r=30, lambda=10, T=15:
    the workload the benchmark times, compared on every document."""
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    want = oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter)
    got = corpus.query(q_ids, q_w, w.lam, w.max_iter)
    assert_parity(got, want, FP32_RTOL, "paper-shaped fp32")
    # the device-resident path (the one the benchmark times) gives the same bits
    dq = wmd.DeviceQuery(corpus, q_ids, q_w)
    dev = dq.run(w.lam, w.max_iter).cpu().numpy()
    import torch
    torch.cuda.synchronize()
    assert np.array_equal(dev[: c.N], got)


def test_paper_exact_shape_all_documents(wmd):
    """The paper's own corpus shape (5000 documents of 10-59 words, about 173k
    nonzeros; queries of 19 and 43 words), every document, FP32 and BF16 K."""
    w = synth.PAPER_EXACT
    vecs = synth.make_vecs(w.V, w.d, synth.embed_seed(w.cfg))
    c = synth.make_corpus(w.V, w.N, w.doc_lo, w.doc_hi, synth.corpus_seed(w.cfg))
    corpus = wmd.Corpus.from_synth(vecs, c)
    for q_ids, q_w in synth.paper_exact_queries():
        want = oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter)
        assert_parity(corpus.query(q_ids, q_w, w.lam, w.max_iter), want, FP32_RTOL,
                      f"paper-exact v_r={len(q_ids)}")
        assert_parity(corpus.query(q_ids, q_w, w.lam, w.max_iter, wmd.PREC_BF16_K), want,
                      BF16_RTOL, f"paper-exact bf16 v_r={len(q_ids)}")
    corpus.close()


def test_large_workload_sampled_documents(wmd):
    """V=100000, N=100000, 20-200 words, v_r=64: sampled documents, FP32 and
    the bfloat16-stored K variant."""
    w = synth.LARGE
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    rng = np.random.default_rng(0)
    lens = np.diff(c.doc_ptr)
    docs = np.unique(np.concatenate([rng.choice(c.N, 400, replace=False),
                                     np.argsort(lens)[-20:], np.argsort(lens)[:20]]))
    want = oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter, docs=docs)
    got = corpus.query(q_ids, q_w, w.lam, w.max_iter)
    assert_parity(got[docs], want, FP32_RTOL, "large fp32")
    got16 = corpus.query(q_ids, q_w, w.lam, w.max_iter, wmd.PREC_BF16_K)
    assert_parity(got16[docs], want, BF16_RTOL, "large bf16")
    assert np.all(np.isfinite(got))


# ---------------------------------------------------------------- query widths and document shapes
@pytest.mark.parametrize("v_r", [1, 2, 7, 8, 9, 16, 17, 31, 32, 33, 48, 49, 64, 65, 96, 97, 100, 128,
                                 129, 192, 193, 200, 256])
def test_query_widths(wmd, v_r):
    """Every padded width class, ragged widths on both sides of each boundary."""
    V, N = 3000, 61
    vecs = synth.make_vecs(V, 300, 40 + v_r)
    c = synth.make_corpus(V, N, 1, 60, 50 + v_r)
    q_ids, q_w = synth.make_query(V, v_r, 60 + v_r)
    corpus = wmd.Corpus.from_synth(vecs, c)
    for T in (0, 1, 15):
        want = oracle(vecs, c, q_ids, q_w, 10.0, T)
        got = corpus.query(q_ids, q_w, 10.0, T)
        assert_parity(got, want, FP32_RTOL, f"v_r={v_r} T={T}")


@pytest.mark.parametrize("v_r,lengths", [
    (30, [1, 2, 95, 96, 97, 150, 192, 193, 385, 700]),    # 1, 2, 4 warps; chunked beyond 384
    (64, [47, 48, 49, 96, 97, 200, 400]),
    (8, [383, 384, 385, 1000]),
    (200, [5, 12, 13, 48, 49, 300]),
    (40, [3, 63, 64, 65, 128, 129, 256, 257, 400]),        # 48-wide tile
    (90, [5, 32, 33, 64, 65, 128, 129, 256, 257, 300]),    # 96-wide tile: 1-8 warps, chunked
    (150, [5, 16, 17, 32, 33, 64, 65, 128, 129, 200]),     # 192-wide tile
])
def test_document_lengths_across_team_sizes(wmd, v_r, lengths):
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
    for T in (1, 15):
        want = oracle(vecs, c, q_ids, q_w, 10.0, T)
        got = corpus.query(q_ids, q_w, 10.0, T)
        assert_parity(got, want, FP32_RTOL, f"lengths v_r={v_r} T={T}")
        got16 = corpus.query(q_ids, q_w, 10.0, T, wmd.PREC_BF16_K)
        assert_parity(got16, want, BF16_RTOL, f"lengths bf16 v_r={v_r} T={T}")


def test_closed_form_cases_on_gpu(wmd):
    """v_r = 1 and single-word documents have closed forms (see the oracle pins)."""
    V = 500
    vecs = synth.make_vecs(V, 300, 77)
    docs = [(np.array([w], np.int32), np.array([1.0], np.float32)) for w in (0, 3, 499)]
    docs.append((np.array([1, 2, 3], np.int32), np.array([0.25, 0.25, 0.5], np.float32)))
    c = synth.corpus_from_docs(V, docs)
    corpus = wmd.Corpus.from_synth(vecs, c)
    import scipy.spatial.distance as ssd
    # one query word
    got = corpus.query([3], [1.0], 10.0, 15)
    M = ssd.cdist(vecs[[3]].astype(np.float64), vecs.astype(np.float64))[0]
    want = np.array([M[0], 0.0, M[499], 0.25 * M[1] + 0.25 * M[2]])
    np.testing.assert_allclose(got, want, rtol=FP32_RTOL, atol=1e-7)
    # single-word documents receive all the query mass
    q_ids = np.array([3, 10, 20], np.int32)
    q_w = np.array([0.5, 0.25, 0.25], np.float32)
    got = corpus.query(q_ids, q_w, 10.0, 15)
    Mq = ssd.cdist(vecs[q_ids].astype(np.float64), vecs.astype(np.float64))
    for j, w_ in enumerate((0, 3, 499)):
        assert abs(got[j] - np.sum(q_w * Mq[:, w_])) <= FP32_RTOL * abs(got[j]) + 1e-7


def test_empty_documents_and_degenerate_corpora(wmd):
    V = 800
    vecs = synth.make_vecs(V, 300, 5)
    c0 = synth.make_corpus(V, 9, 3, 30, 6)
    docs = _docs(c0)
    docs.insert(0, (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    docs.insert(5, (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    c = synth.corpus_from_docs(V, docs)
    q_ids, q_w = synth.make_query(V, 12, 7)
    corpus = wmd.Corpus.from_synth(vecs, c)
    for T in (0, 1, 15):
        want = oracle(vecs, c, q_ids, q_w, 10.0, T)
        got = corpus.query(q_ids, q_w, 10.0, T)
        assert_parity(got, want, FP32_RTOL, f"empty docs T={T}")
    # a corpus without any nonzero and one without documents
    cz = synth.corpus_from_docs(V, [(np.zeros(0, np.int32), np.zeros(0, np.float32))] * 3)
    got = wmd.Corpus.from_synth(vecs, cz).query(q_ids, q_w, 10.0, 5)
    assert np.all(np.isnan(got))
    cn = synth.corpus_from_docs(V, [])
    assert wmd.Corpus.from_synth(vecs, cn).query(q_ids, q_w, 10.0, 5).shape == (0,)


def test_zero_weight_query_words_are_dropped(wmd):
    V = 1000
    vecs = synth.make_vecs(V, 300, 8)
    c = synth.make_corpus(V, 20, 5, 40, 9)
    q_ids, q_w = synth.make_query(V, 10, 10)
    corpus = wmd.Corpus.from_synth(vecs, c)
    base = corpus.query(q_ids, q_w, 10.0, 15)
    ids2 = np.concatenate([[V - 1], q_ids, [V - 2]]).astype(np.int32)
    w2 = np.concatenate([[0.0], q_w, [0.0]]).astype(np.float32)
    np.testing.assert_array_equal(corpus.query(ids2, w2, 10.0, 15), base)


def test_odd_embedding_width_and_other_lambdas(wmd):
    V = 1500
    # (8, 10): few dimensions put some distinct words close together, where the
    # GEMM form |a|^2 + |b|^2 - 2ab loses digits to cancellation (Sec. 5); the
    # cdist kernels recompute those near pairs by direct differences
    for d, lam, tol in [(37, 3.0, FP32_RTOL), (8, 10.0, FP32_RTOL), (512, 20.0, FP32_RTOL)]:
        vecs = synth.make_vecs(V, d, d)
        c = synth.make_corpus(V, 33, 4, 50, d + 1)
        q_ids, q_w = synth.make_query(V, 21, d + 2)
        corpus = wmd.Corpus.from_synth(vecs, c)
        want = oracle(vecs, c, q_ids, q_w, lam, 15)
        got = corpus.query(q_ids, q_w, lam, 15)
        assert_parity(got, want, tol, f"d={d} lambda={lam}")


def test_invalid_arguments_return_errors(wmd):
    V = 100
    vecs = synth.make_vecs(V, 8, 1)
    c = synth.make_corpus(V, 4, 2, 5, 2)
    corpus = wmd.Corpus.from_synth(vecs, c)
    for args, st in [(([1], [1.0], 0.0, 5), wmd.WMD_ERR_INVALID_ARG),
                     (([1], [1.0], float("nan"), 5), wmd.WMD_ERR_INVALID_ARG),
                     (([1], [1.0], 1.0, -1), wmd.WMD_ERR_INVALID_ARG),
                     (([1], [0.0], 1.0, 5), wmd.WMD_ERR_INVALID_ARG),
                     (([100], [1.0], 1.0, 5), wmd.WMD_ERR_INVALID_ARG)]:
        with pytest.raises(wmd.WMDError) as e:
            corpus.query(*args)
        assert e.value.status == st
    import torch
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(wmd.WMDError):
        corpus.query_device(torch.zeros(1, dtype=torch.int32, device="cuda"),
                            torch.ones(1, device="cuda"), 1, 1.0, 1, wmd.PREC_FP32, ws, 16,
                            torch.empty(4, dtype=torch.float64, device="cuda"))


def test_out_of_range_device_id_gives_nan_not_a_fault(wmd):
    import torch
    V = 200
    vecs = synth.make_vecs(V, 16, 1)
    c = synth.make_corpus(V, 5, 2, 9, 2)
    corpus = wmd.Corpus.from_synth(vecs, c)
    ids = torch.tensor([3, V + 5], dtype=torch.int32, device="cuda")
    w = torch.tensor([0.5, 0.5], device="cuda")
    nb = corpus.workspace_bytes(2)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.empty(c.N, dtype=torch.float64, device="cuda")
    corpus.query_device(ids, w, 2, 10.0, 5, wmd.PREC_FP32, ws, nb, out)
    torch.cuda.synchronize()
    assert torch.isnan(out).all()


# ---------------------------------------------------------------- K1 directly
def _active_words(c):
    return np.flatnonzero(np.diff(c.row_ptr))


def _workspace_k(wmd, corpus, dq, VR, prec):
    """Padded weights r, lambda and K (U x VR) read back from the workspace
    after the cdist stage."""
    import torch
    U = corpus.U
    esz = 2 if prec == wmd.PREC_BF16_K else 4
    k_off = ((VR + 1) * 4 + 255) // 256 * 256
    raw = dq.ws.cpu()
    r_lam = raw[: (VR + 1) * 4].view(torch.float32).numpy()
    dt = torch.bfloat16 if esz == 2 else torch.float32
    K = raw[k_off:k_off + U * VR * esz].view(dt).float().numpy().reshape(U, VR)
    return r_lam[:VR], float(r_lam[VR]), K


@pytest.mark.parametrize("kernel", ["tc", "simt"])
@pytest.mark.parametrize("v_r", [5, 16, 30, 64, 100])
def test_cdist_kernel_matrix_elementwise(wmd, monkeypatch, kernel, v_r):
    """K = exp(-lambda M) against the oracle's FP64 distances, for the
    tensor-core (fp16 pairs) and the CUDA-core kernel; the query's own words give
    K = 1 exactly; padding columns are 0; r and lambda land next to K."""
    import torch
    if kernel == "simt":
        monkeypatch.setenv("WMD_CDIST_KERNEL", "simt")
    else:
        monkeypatch.delenv("WMD_CDIST_KERNEL", raising=False)
    V, lam = 5000, 10.0
    vecs = synth.make_vecs(V, 300, 11)
    c = synth.make_corpus(V, 300, 5, 60, 12)
    q_ids, q_w = synth.make_query(V, v_r, 13)
    corpus = wmd.Corpus.from_synth(vecs, c)
    # float32 tolerance from the arithmetic: m^2 = |a|^2 + |b|^2 - 2 a.b carries
    # a few ulps of |a|^2 + |b|^2 ~ 2 (about 1e-6 absolute); distinct N(0, 1/d)
    # words are >= ~0.5 apart, so |dm| <= 1e-6 and |dK / K| = lambda |dm| <= 1e-5.
    # bfloat16 storage adds its 2^-9 rounding.
    for prec, rtol in [(wmd.PREC_FP32, 1e-5), (wmd.PREC_BF16_K, 1e-2)]:
        dq = wmd.DeviceQuery(corpus, q_ids, q_w, prec)
        corpus.build_kernel_matrix(dq.ids, dq.w, dq.v_r, lam, prec, dq.ws, dq.ws_bytes)
        torch.cuda.synchronize()
        VR = 8
        while VR < v_r:
            VR *= 2
        r, lam_ws, K = _workspace_k(wmd, corpus, dq, VR, prec)
        assert lam_ws == np.float32(lam)
        np.testing.assert_array_equal(r[:v_r], dq.w.cpu().numpy())
        assert np.all(r[v_r:] == 0)
        words = _active_words(c)
        M = orc.cdist(vecs, q_ids, words).T                    # U x v_r
        Kw = np.exp(-lam * M)
        np.testing.assert_allclose(K[:, :v_r], Kw, rtol=rtol, atol=0)
        assert np.all(K[:, v_r:] == 0)
        own = np.isin(words, q_ids)
        rows, cols = np.nonzero(words[:, None] == q_ids[None, :])
        assert np.all(K[rows, cols] == 1.0)
        assert own.sum() == len(rows)


def test_cdist_tc_rows_of_mixed_magnitude(wmd, monkeypatch):
    """The tensor-core cdist scales every vocabulary row by its own power of
    two before splitting it into fp16 hi and lo parts: rows whose magnitudes
    span 12 decades keep float32-grade distances.  Bound per element from the
    arithmetic: the pair product loses at most ~2^-21 |a| |b| and m^2 a few
    float32 ulps of |a|^2 + |b|^2, so |dm| <= 1e-5 (|a|^2 + |b|^2) / (2 m)
    (or the square root of that numerator when m is smaller) and
    |dK| <= K (lambda |dm| + 2.4e-7), the last term for expf and the float32
    rounding of K itself (4 ulps: K = 1 - 1e-8 is stored as 1)."""
    import torch
    monkeypatch.delenv("WMD_CDIST_KERNEL", raising=False)
    V, d, v_r = 3000, 64, 16
    rng = np.random.default_rng(23)
    vecs = synth.make_vecs(V, d, 21) * (10.0 ** rng.uniform(-6, 6, size=(V, 1))).astype(np.float32)
    vecs = vecs.astype(np.float32)
    c = synth.make_corpus(V, 200, 5, 40, 22)
    q_ids, q_w = synth.make_query(V, v_r, 24)
    corpus = wmd.Corpus.from_synth(vecs, c)
    words = _active_words(c)
    M = orc.cdist(vecs, q_ids, words).T                    # U x v_r, float64
    lam = float(3.0 / np.median(M))
    dq = wmd.DeviceQuery(corpus, q_ids, q_w, wmd.PREC_FP32)
    corpus.build_kernel_matrix(dq.ids, dq.w, dq.v_r, lam, wmd.PREC_FP32, dq.ws, dq.ws_bytes)
    torch.cuda.synchronize()
    _, _, K = _workspace_k(wmd, corpus, dq, 16, wmd.PREC_FP32)
    a2 = np.sum(vecs[words].astype(np.float64) ** 2, axis=1)[:, None]
    b2 = np.sum(vecs[q_ids].astype(np.float64) ** 2, axis=1)[None, :]
    dm2 = 1e-5 * (a2 + b2)
    dm = np.where(M * M > dm2, dm2 / (2 * np.maximum(M, 1e-300)), np.sqrt(dm2))
    Kw = np.exp(-lam * M)
    err = np.abs(K[:, :v_r].astype(np.float64) - Kw)
    bound = Kw * (np.expm1(lam * dm) + 2.4e-7) + 1e-37
    assert np.all(err <= bound), f"worst excess {np.max(err / bound):.3g}"
    # and a non-trivial share of K is well above underflow
    assert np.mean(Kw > 1e-6) > 0.05


@pytest.mark.parametrize("kernel", ["tc", "simt"])
def test_paper_shaped_with_both_cdist_kernels(wmd, monkeypatch, kernel):
    if kernel == "simt":
        monkeypatch.setenv("WMD_CDIST_KERNEL", "simt")
    else:
        monkeypatch.delenv("WMD_CDIST_KERNEL", raising=False)
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    rng = np.random.default_rng(5)
    docs = np.sort(rng.choice(c.N, 300, replace=False))
    want = oracle(vecs, c, q_ids, q_w, w.lam, w.max_iter, docs=docs)
    got = corpus.query(q_ids, q_w, w.lam, w.max_iter)
    assert_parity(got[docs], want, FP32_RTOL, f"paper-shaped fp32 {kernel}")


# ---------------------------------------------------------------- fused-loop tile variants
@pytest.mark.parametrize("v_r", [6, 16, 30, 40, 64, 80, 100, 150, 200])
def test_every_loop_variant_matches_oracle(wmd, v_r):
    """Each register-tile variant of each width class gives the oracle's
    values (documents long enough for teams of 1, 2 and 4 warps and for the
    chunked path), and the autotuner picks one of them."""
    V = 4000
    vecs = synth.make_vecs(V, 300, 500 + v_r)
    rng = np.random.default_rng(v_r)
    lengths = [1, 7, 20, 40, 48, 64, 65, 96, 97, 130, 192, 193, 260, 400]
    docs = []
    for n in lengths:
        ids = np.sort(rng.choice(V, n, replace=False)).astype(np.int32)
        wts = rng.random(n) + 0.05
        docs.append((ids, (wts / wts.sum()).astype(np.float32)))
    c = synth.corpus_from_docs(V, docs)
    q_ids, q_w = synth.make_query(V, v_r, 600 + v_r)
    corpus = wmd.Corpus.from_synth(vecs, c)
    want = oracle(vecs, c, q_ids, q_w, 10.0, 15)
    n_var = wmd.loop_variant_count(v_r)
    assert n_var >= 1
    for var in range(n_var):
        corpus.set_loop_variant(v_r, var)
        assert_parity(corpus.query(q_ids, q_w, 10.0, 15), want, FP32_RTOL, f"v_r={v_r} variant {var}")
        corpus.set_loop_variant(v_r, var, wmd.PREC_BF16_K)
        assert_parity(corpus.query(q_ids, q_w, 10.0, 15, wmd.PREC_BF16_K), want, BF16_RTOL,
                      f"bf16 v_r={v_r} variant {var}")
    chosen = corpus.autotune(q_ids, q_w, 10.0, 15)
    assert 0 <= chosen < n_var
    assert_parity(corpus.query(q_ids, q_w, 10.0, 15), want, FP32_RTOL, "after autotune")
    with pytest.raises(wmd.WMDError):
        corpus.set_loop_variant(v_r, n_var)


# ---------------------------------------------------------------- partitions (team sizes)
@pytest.mark.parametrize("v_r", [6, 30, 40, 64, 80, 100, 150, 200])
def test_every_partition_matches_oracle(wmd, v_r):
    """Every partition of the documents into teams (fill 50, 75, 100, 200:
    spread over more warps, the default, or long documents re-read from L2
    by fewer warps) with every tile variant gives the oracle's values, and
    the autotuner's choice of variant and partition too."""
    V = 4000
    vecs = synth.make_vecs(V, 300, 700 + v_r)
    rng = np.random.default_rng(800 + v_r)
    lengths = [1, 2, 7, 20, 33, 48, 49, 64, 65, 96, 97, 130, 192, 193, 260, 400, 800]
    docs = []
    for n in lengths:
        ids = np.sort(rng.choice(V, n, replace=False)).astype(np.int32)
        wts = rng.random(n) + 0.05
        docs.append((ids, (wts / wts.sum()).astype(np.float32)))
    c = synth.corpus_from_docs(V, docs)
    q_ids, q_w = synth.make_query(V, v_r, 900 + v_r)
    corpus = wmd.Corpus.from_synth(vecs, c)
    for T in (0, 15):
        want = oracle(vecs, c, q_ids, q_w, 10.0, T)
        for var in range(wmd.loop_variant_count(v_r)):
            corpus.set_loop_variant(v_r, var)
            corpus.set_loop_variant(v_r, var, wmd.PREC_BF16_K)
            for fill in (50, 75, 100, 200):
                corpus.set_loop_partition(v_r, var, fill)
                assert corpus.loop_partition(v_r, var) == fill
                assert_parity(corpus.query(q_ids, q_w, 10.0, T), want, FP32_RTOL,
                              f"v_r={v_r} T={T} variant {var} fill {fill}")
                assert_parity(corpus.query(q_ids, q_w, 10.0, T, wmd.PREC_BF16_K), want, BF16_RTOL,
                              f"bf16 v_r={v_r} T={T} variant {var} fill {fill}")
    want = oracle(vecs, c, q_ids, q_w, 10.0, 15)
    chosen = corpus.autotune(q_ids, q_w, 10.0, 15)
    assert corpus.loop_variant(v_r) == chosen
    assert corpus.loop_partition(v_r, chosen) in (50, 75, 100, 200)
    assert_parity(corpus.query(q_ids, q_w, 10.0, 15), want, FP32_RTOL, "after autotune")
    for bad in (0, 60, 101, 400):
        with pytest.raises(wmd.WMDError):
            corpus.set_loop_partition(v_r, 0, bad)
    with pytest.raises(wmd.WMDError):
        corpus.set_loop_partition(v_r, wmd.loop_variant_count(v_r), 100)
    assert corpus.loop_partition(v_r, 99) == -1
    corpus.close()


def test_measured_fp32_peak_is_plausible(wmd):
    """wmd_measure_fp32_peak (the fused loop's roofline denominator) lies
    below the unit-count bound (SMs x 128 FP32 lanes x 2 flop x 2.2 GHz, above
    any GB300 clock) and not far under it; an invalid device is refused."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    for packed in (True, False):
        t = wmd.measure_fp32_peak(0, packed)
        assert 0.3 * bound < t < bound, (packed, t, bound)
    with pytest.raises(wmd.WMDError):
        wmd.measure_fp32_peak(torch.cuda.device_count(), True)
