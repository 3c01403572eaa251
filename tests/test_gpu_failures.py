"""Failure detection and the library's options on the GPU.

The device-side failures are made without faulting anything: a wait limit of
a few clock cycles makes the tensor-core cdist kernel's bounded waits run out
(its TMA copies and MMAs are still retired before the CTA returns), and a
large lambda pushes lambda * M past the float32 range of K = exp(-lambda M).
Each test then checks that the error is reported for the query that caused it
and for no other: the error words are per query (per workspace, per batched
query), so the next query on the same corpus, workspace or server is clean.
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


@pytest.fixture(scope="module")
def small():
    V = 3000
    vecs = synth.make_vecs(V, 64, 31)
    c = synth.make_corpus(V, 120, 5, 60, 32)
    qs = [synth.make_query(V, n, 33 + n) for n in (7, 19, 30, 45)]
    return vecs, c, qs


def _oracle(vecs, c, q, lam, T=15):
    return orc.sinkhorn_wmd_sparse(q[0], q[1], c.row_ptr, c.doc_idx, c.val, c.N, vecs, lam, T)


def _close(got, want, rtol=FP32_RTOL):
    got, want = np.asarray(got), np.asarray(want)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    rel = np.abs(got[ok] - want[ok]) / np.maximum(np.abs(want[ok]), 1e-7)
    assert rel.max() <= rtol, rel.max()


def test_cdist_wait_timeout_then_clean_query_on_the_same_corpus(wmd, small):
    import torch
    vecs, c, qs = small
    corpus = wmd.Corpus.from_synth(vecs, c, wait_limit_cycles=1)
    assert corpus.cdist_kernel.startswith("tensor cores")
    q = qs[2]
    # host path: the timeout is reported and no result is returned
    with pytest.raises(wmd.WMDError) as e:
        corpus.query(q[0], q[1], 10.0, 15)
    assert e.value.status == wmd.WMD_ERR_TIMEOUT
    assert "timed out" in str(e.value)
    # device path: NaN for every document, written by the loop kernel
    dq = wmd.DeviceQuery(corpus, q[0], q[1])
    dq.out.fill_(0.0)
    out = dq.run(10.0, 15).cpu().numpy()[: c.N]
    torch.cuda.synchronize()
    assert np.isnan(out).all()
    # the same corpus, host path and workspace: clean again with the default limit
    corpus.set_wait_limit(0)
    want = _oracle(vecs, c, q, 10.0)
    _close(corpus.query(q[0], q[1], 10.0, 15), want)
    _close(corpus.query(q[0], q[1], 10.0, 15), want)   # second call: captured graph
    _close(dq.run(10.0, 15).cpu().numpy()[: c.N], want)
    corpus.close()


def test_server_timeout_fails_only_its_own_batches(wmd, small):
    vecs, c, qs = small
    corpus = wmd.Corpus.from_synth(vecs, c)
    alone = [corpus.query(q[0], q[1], 10.0, 15) for q in qs]
    corpus.set_wait_limit(1)
    srv = wmd.Server(corpus, max_batch=4, slots=2)
    try:
        ts = [srv.submit(q[0], q[1], 10.0, 15) for q in qs]
        for t in ts:
            with pytest.raises(wmd.WMDError) as e:
                srv.poll(t, timeout_us=30_000_000)
            assert e.value.status == wmd.WMD_ERR_TIMEOUT
    finally:
        srv.close()
    corpus.set_wait_limit(0)
    srv = wmd.Server(corpus, max_batch=4, slots=2)
    try:
        ts = [srv.submit(q[0], q[1], 10.0, 15) for q in qs]
        for t, a in zip(ts, alone):
            np.testing.assert_array_equal(srv.poll(t, timeout_us=30_000_000), a)
    finally:
        srv.close()
    corpus.close()


def test_range_limit_is_reported_per_query(wmd, small):
    """lambda * M >= 87.3 would make K subnormal: WMD_ERR_RANGE on the host
    paths and NaN on the device path, for that query only."""
    import torch
    vecs, c, qs = small
    corpus = wmd.Corpus.from_synth(vecs, c)
    q = qs[1]
    # distinct N(0, 1/d) words are about sqrt(2) apart: lambda = 100 leaves the range
    with pytest.raises(wmd.WMDError) as e:
        corpus.query(q[0], q[1], 100.0, 15)
    assert e.value.status == wmd.WMD_ERR_RANGE
    dq = wmd.DeviceQuery(corpus, q[0], q[1])
    out = dq.run(100.0, 15).cpu().numpy()[: c.N]
    torch.cuda.synchronize()
    assert np.isnan(out).all()
    # the same workspace and corpus at lambda = 10: oracle results
    want = _oracle(vecs, c, q, 10.0)
    _close(dq.run(10.0, 15).cpu().numpy()[: c.N], want)
    _close(corpus.query(q[0], q[1], 10.0, 15), want)
    # a batch reports the failed query; the server fails that request alone
    with pytest.raises(wmd.WMDError) as e:
        corpus.query_batch([qs[0], q, qs[2]], [10.0, 100.0, 10.0], 15)
    assert e.value.status == wmd.WMD_ERR_RANGE and "query 1" in str(e.value)
    alone = [corpus.query(x[0], x[1], 10.0, 15) for x in qs]
    srv = wmd.Server(corpus, max_batch=8, slots=1)
    try:
        ts = [srv.submit(x[0], x[1], 100.0 if k == 1 else 10.0, 15) for k, x in enumerate(qs)]
        for k, t in enumerate(ts):
            if k == 1:
                with pytest.raises(wmd.WMDError) as e:
                    srv.poll(t, timeout_us=30_000_000)
                assert e.value.status == wmd.WMD_ERR_RANGE
            else:
                np.testing.assert_array_equal(srv.poll(t, timeout_us=30_000_000), alone[k])
    finally:
        srv.close()
    corpus.close()


def test_refused_device_call_writes_nothing(wmd, small):
    """Every argument is checked before the first launch: a call refused for
    a NULL output leaves the workspace untouched."""
    import torch
    vecs, c, qs = small
    corpus = wmd.Corpus.from_synth(vecs, c)
    dq = wmd.DeviceQuery(corpus, qs[0][0], qs[0][1])
    dq.ws.fill_(0x5A)
    torch.cuda.synchronize()
    with pytest.raises(wmd.WMDError) as e:
        corpus.query_device(dq.ids, dq.w, dq.v_r, 10.0, 15, wmd.PREC_FP32, dq.ws, dq.ws_bytes,
                            None)
    assert e.value.status == wmd.WMD_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert bool((dq.ws == 0x5A).all())
    corpus.close()


def test_options_cdist_kernel_and_graphs(wmd, small):
    """The CUDA-core cdist is an explicit option, reported by the corpus; both
    kernels and both launch modes give oracle results."""
    vecs, c, qs = small
    q = qs[3]
    want = _oracle(vecs, c, q, 10.0)
    for kw, kernel in [({}, "tensor cores"), ({"cdist_kernel": wmd.CDIST_CUDA_CORES}, "CUDA cores"),
                       ({"use_graphs": False}, "tensor cores")]:
        corpus = wmd.Corpus.from_synth(vecs, c, **kw)
        assert corpus.cdist_kernel.startswith(kernel)
        for _ in range(3):
            _close(corpus.query(q[0], q[1], 10.0, 15), want)
        res = corpus.query_batch(qs, 10.0, 15)
        _close(res[3], want)
        corpus.close()


def test_autotune_cache_round_trip(wmd, small, tmp_path):
    vecs, c, qs = small
    path = tmp_path / "tune.txt"
    corpus = wmd.Corpus.from_synth(vecs, c, autotune_cache=str(path))
    chosen = corpus.autotune(qs[2][0], qs[2][1], 10.0, 15)
    v_r = len(qs[2][0])
    assert corpus.loop_variant(v_r) == chosen
    corpus.close()
    lines = path.read_text().splitlines()
    assert lines and lines[-1].startswith("wmd-loop ")
    fields = lines[-1].split()
    assert len(fields) == 10 and int(fields[-2]) == chosen and int(fields[-1]) in (50, 75, 100, 200)
    # a corpus of the same shape starts from the recorded choice; a forced
    # entry for the other variant and partition wins (last line); malformed
    # lines and invalid partitions are skipped
    other = 1 - chosen
    fields[-2], fields[-1] = str(other), "200"
    bad_fill = fields[:-1] + ["60"]
    path.write_text("\n".join(lines + ["garbage line", " ".join(fields), " ".join(bad_fill)]) + "\n")
    corpus = wmd.Corpus.from_synth(vecs, c, autotune_cache=str(path))
    assert corpus.loop_variant(v_r) == other
    assert corpus.loop_partition(v_r, other) == 200
    _close(corpus.query(qs[2][0], qs[2][1], 10.0, 15), _oracle(vecs, c, qs[2], 10.0))
    corpus.close()
    # a line without a partition (variant only) keeps fill = 100
    path.write_text(" ".join(fields[:-1]) + "\n")
    corpus = wmd.Corpus.from_synth(vecs, c, autotune_cache=str(path))
    assert corpus.loop_variant(v_r) == other
    assert corpus.loop_partition(v_r, other) == 100
    corpus.close()
    # another corpus shape ignores the file
    c2 = synth.make_corpus(vecs.shape[0], 50, 5, 60, 77)
    corpus = wmd.Corpus.from_synth(vecs, c2, autotune_cache=str(path))
    assert corpus.loop_variant(v_r) == 0
    corpus.close()
