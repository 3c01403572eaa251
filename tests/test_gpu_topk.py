"""k nearest documents (wmd_topk, wmd_query_device_topk) against the oracle.

The selection orders WMD values with ties to the lower document id and NaN
last, so the answer on a given WMD vector is unique: the GPU's ids and values
must equal the oracle's selection from the same vector bit for bit.  Against
the FP64 oracle's own WMD values the k nearest may differ only where two
documents lie within the WMD tolerance (1e-5 relative) of each other.
"""
import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wmd():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import wmd as w
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return w


def _select(wmd, values, k):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(values, np.float64)).cuda()
    idx = torch.full((max(k, 1),), -5, dtype=torch.int64, device="cuda")
    val = torch.full((max(k, 1),), -5.0, dtype=torch.float64, device="cuda")
    wmd.topk(d, values.size, k, idx, val)
    torch.cuda.synchronize()
    return idx.cpu().numpy()[:k], val.cpu().numpy()[:k]


def _values(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "wmd":                      # WMD-like: around 1.2-1.5, all distinct
        return 1.2 + 0.3 * rng.random(n)
    if kind == "ties":                     # few distinct values, signed zeros, NaN, inf
        v = rng.choice([1.5, 1.25, 0.0, -0.0, 2.0, np.nan, np.inf, 1.25], n)
        return v.astype(np.float64)
    if kind == "dense":                    # a few ulps apart: several digit passes, many ties
        return 1.0 + rng.integers(0, 3000, n) * 2.0 ** -50
    if kind == "nan":
        return np.full(n, np.nan)
    if kind == "equal":
        return np.full(n, 1.375)
    raise ValueError(kind)


@pytest.mark.parametrize("n", [1, 2, 100, 511, 512, 513, 1023, 1024, 1025, 5000, 12288, 12289,
                               16384, 16385, 50_000, 131_072, 131_073, 200_000, 262_144, 262_145])
@pytest.mark.parametrize("kind", ["wmd", "ties", "dense"])
def test_selection_is_bit_exact(wmd, n, kind):
    """Every selection kernel at its edges: keys in registers of one CTA (N <=
    16384, k <= 256), of a thread-block cluster (N up to 8 or 16 CTAs x 16384,
    k <= 256), and the shared-memory / streamed radix select otherwise."""
    v = _values(n, kind, n)
    for k in sorted({1, min(7, n), min(100, n), min(256, n), min(257, n), min(1024, n)}):
        ids, vals = _select(wmd, v, k)
        want_ids, want_vals = orc.nearest_documents(v, k)
        assert ids.tolist() == want_ids.tolist(), f"n={n} k={k} {kind}"
        assert np.array_equal(vals.view(np.int64), want_vals.view(np.int64)), f"n={n} k={k} {kind}"


@pytest.mark.parametrize("kind", ["nan", "equal"])
def test_all_equal_values_give_the_lowest_ids(wmd, kind):
    for n in (50, 600, 3000, 16384, 20000, 150_000):
        v = _values(n, kind, 0)
        k = min(64, n - 1)
        ids, vals = _select(wmd, v, k)
        assert ids.tolist() == list(range(k))
        assert np.array_equal(vals, v[:k], equal_nan=True)


def test_k_out_of_range_is_rejected(wmd):
    v = _values(10, "wmd", 1)
    for k in (11, -1, 2000):
        with pytest.raises(wmd.WMDError) as e:
            _select(wmd, v, k)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
    ids, vals = _select(wmd, v, 0)
    assert ids.size == 0


def test_query_topk_paper_shaped(wmd):
    """The retrieval call on the paper-shaped workload: the ids are the
    selection from its own WMD output, and agree with the FP64 oracle's
    nearest documents up to documents within the WMD tolerance of the k-th."""
    import torch
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    q_ids, q_w = qs[0]
    dq = wmd.DeviceQuery(corpus, q_ids, q_w)
    k = 100
    idx = torch.empty(k, dtype=torch.int64, device="cuda")
    val = torch.empty(k, dtype=torch.float64, device="cuda")
    corpus.query_device_topk(dq.ids, dq.w, dq.v_r, w.lam, w.max_iter, wmd.PREC_FP32, dq.ws,
                             dq.ws_bytes, dq.out, k, idx, val)
    torch.cuda.synchronize()
    got = dq.out[: c.N].cpu().numpy()
    ids, vals = idx.cpu().numpy(), val.cpu().numpy()
    want_ids, _ = orc.nearest_documents(got, k)
    assert ids.tolist() == want_ids.tolist()
    assert np.array_equal(vals, got[ids])

    ref = orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N, vecs, w.lam,
                                  w.max_iter)
    ref_ids, ref_vals = orc.nearest_documents(ref, k)
    kth = ref_vals[-1]
    for j in set(ids.tolist()) ^ set(ref_ids.tolist()):
        assert abs(ref[j] - kth) <= 2e-5 * kth, f"document {j} is not a near-tie of the k-th"
