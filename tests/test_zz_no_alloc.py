"""The workspace-free entry point (wmd_query_device_noalloc) gives the same
WMD values as the workspace entry point (wmd_query_device).

It exists for callers that may not allocate device memory; its scratch is a
fixed array inside the library that every call reuses, so two calls in a row
are checked (the second one must not see stale data from the first), and a
query that needs more scratch than the array holds must be refused.  This file
is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


def _close(got, want, rtol):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    rel = np.abs(got[~nan] - want[~nan]) / np.maximum(np.abs(want[~nan]), 1e-7)
    assert rel.size == 0 or rel.max() <= rtol, rel.max()


def test_noalloc_entry_point_matches_workspace_entry_point():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    import torch
    from paper_2005_06727_gb300 import wmd

    assert torch.cuda.is_available()
    w = synth.PAPER
    vecs, c, qs = synth.make_workload(w)
    corpus = wmd.Corpus.from_synth(vecs, c)
    dev = torch.device("cuda", corpus.device)
    # two different queries in a row: the second reuses the shared scratch
    queries = [qs[0], synth.make_query(w.V, 20, 4242)]
    for q_ids, q_w in queries:
        ids = torch.from_numpy(np.ascontiguousarray(q_ids)).to(dev)
        wts = torch.from_numpy(np.ascontiguousarray(q_w)).to(dev)
        v_r = int(ids.numel())
        for prec, rtol in [(wmd.PREC_FP32, FP32_RTOL), (wmd.PREC_BF16_K, FP32_RTOL)]:
            ws_bytes = corpus.workspace_bytes(v_r, prec)
            ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
            ref = torch.empty(c.N, dtype=torch.float64, device=dev)
            corpus.query_device(ids, wts, v_r, w.lam, w.max_iter, prec, ws, ws_bytes, ref)
            out = torch.full((c.N,), -1.0, dtype=torch.float64, device=dev)
            wmd.query_device_noalloc(corpus, ids, wts, v_r, w.lam, w.max_iter, prec, out)
            torch.cuda.synchronize()
            _close(out.cpu().numpy(), ref.cpu().numpy(), rtol)
            assert np.all(np.isfinite(out.cpu().numpy()))

    # more scratch than the built-in array holds is refused, not truncated
    big_ids, big_w = synth.make_query(w.V, 128, 77)
    ids = torch.from_numpy(big_ids).to(dev)
    wts = torch.from_numpy(big_w).to(dev)
    assert corpus.workspace_bytes(128) > 16 << 20
    out = torch.empty(c.N, dtype=torch.float64, device=dev)
    with pytest.raises(wmd.WMDError) as e:
        wmd.query_device_noalloc(corpus, ids, wts, 128, w.lam, w.max_iter, wmd.PREC_FP32, out)
    assert e.value.status == wmd.WMD_ERR_UNSUPPORTED
    corpus.close()
