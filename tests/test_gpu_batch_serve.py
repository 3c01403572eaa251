"""Batched and served queries (GPU): every query's result is bit-identical to
the same query run alone through wmd_query, whatever else shares its batch or
the server's mix; and the oracle agrees on sampled queries."""
import time

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
    return w


@pytest.fixture(scope="module")
def setup(wmd):
    V, N = 6000, 400
    vecs = synth.make_vecs(V, 300, 101)
    c = synth.make_corpus(V, N, 5, 80, 102)
    corpus = wmd.Corpus.from_synth(vecs, c)
    rng = np.random.default_rng(7)
    widths = [1, 3, 8, 9, 16, 17, 30, 32, 33, 64, 65, 100, 128, 129, 200, 256, 80, 96, 97, 150, 192, 193,
              20, 40, 48, 49]
    queries = [synth.make_query(V, int(vr), 300 + i) for i, vr in enumerate(widths)]
    queries += [synth.make_query(V, int(rng.integers(5, 129)), 400 + i) for i in range(12)]
    return vecs, c, corpus, queries


def _alone(corpus, queries, lam, T, prec):
    return np.stack([corpus.query(q[0], q[1], lam, T, prec) for q in queries])


@pytest.mark.parametrize("prec_name", ["fp32", "bf16"])
def test_batch_equals_alone_bitwise(wmd, setup, prec_name):
    vecs, c, corpus, queries = setup
    prec = wmd.PREC_FP32 if prec_name == "fp32" else wmd.PREC_BF16_K
    alone = _alone(corpus, queries, 10.0, 15, prec)
    batch = corpus.query_batch(queries, 10.0, 15, prec)
    assert np.array_equal(batch, alone)
    # again with the same shape: the captured graph is replayed
    batch2 = corpus.query_batch(queries, 10.0, 15, prec)
    assert np.array_equal(batch2, alone)


def test_graph_replay_with_new_words_and_lambdas(wmd, setup):
    vecs, c, corpus, queries = setup
    lams = np.linspace(3.0, 12.0, len(queries)).astype(np.float32)
    first = corpus.query_batch(queries, lams, 7)
    # same widths, different words: the replayed graph must read the new words
    other = [synth.make_query(c.V, len(q[0]), 900 + i) for i, q in enumerate(queries)]
    got = corpus.query_batch(other, lams, 7)
    want = np.stack([corpus.query(q[0], q[1], float(l), 7) for q, l in zip(other, lams)])
    assert np.array_equal(got, want)
    assert not np.array_equal(first, got)


def test_query_into_pinned_output_buffers(wmd, setup):
    """wmd_query writes straight into a caller buffer that is pinned and mapped
    (and through its own staging block otherwise): every route, first use and
    graph replay alike, gives the same bits."""
    torch = pytest.importorskip("torch")
    _, c, corpus, queries = setup
    q_ids, q_w = queries[6]
    ref = corpus.query(q_ids, q_w, 10.0, 15)  # pageable output
    pinned = [torch.empty(c.N, dtype=torch.float64).pin_memory().numpy() for _ in range(2)]
    for _ in range(3):  # eager, capture, replay
        for buf in pinned:
            buf.fill(np.nan)
            corpus.query(q_ids, q_w, 10.0, 15, out=buf)
            assert np.array_equal(buf, ref)
    again = corpus.query(q_ids, q_w, 10.0, 15)
    assert np.array_equal(again, ref)
    # read-only query arrays and a strided view are marshalled by copy or address
    ro_ids, ro_w = q_ids.copy(), q_w.copy()
    ro_ids.setflags(write=False)
    ro_w.setflags(write=False)
    assert np.array_equal(corpus.query(ro_ids, ro_w, 10.0, 15), ref)
    strided = np.repeat(q_ids, 2)[::2]
    assert not strided.flags.c_contiguous
    assert np.array_equal(corpus.query(strided, q_w, 10.0, 15), ref)
    # an output buffer the library could not fill in place is refused
    for bad in (np.empty(c.N, np.float32), np.empty(2 * c.N)[::2], np.empty(c.N - 1)):
        with pytest.raises(ValueError):
            corpus.query(q_ids, q_w, 10.0, 15, out=bad)


def test_batch_against_oracle(wmd, setup):
    vecs, c, corpus, queries = setup
    sel = [0, 6, 11, 15, 17, 19, 20, 23, 24, 28]  # v_r 1, 30, 100, 256, 96, 150, 192, 40, 48, random
    got = corpus.query_batch([queries[i] for i in sel], 10.0, 15)
    for row, i in enumerate(sel):
        want = orc.sinkhorn_wmd_sparse(queries[i][0], queries[i][1], c.row_ptr, c.doc_idx, c.val,
                                       c.N, vecs, 10.0, 15)
        rel = np.abs(got[row] - want) / np.maximum(np.abs(want), 1e-7)
        assert rel.max() <= FP32_RTOL, (i, rel.max())


def test_batch_input_errors(wmd, setup):
    vecs, c, corpus, queries = setup
    with pytest.raises(wmd.WMDError) as e:
        corpus.query_batch([queries[0], (np.array([c.V + 1], np.int32), np.array([1.0], np.float32))], 10.0, 5)
    assert e.value.status == wmd.WMD_ERR_INVALID_ARG
    with pytest.raises(wmd.WMDError):
        corpus.query_batch([queries[0]], -1.0, 5)
    assert corpus.query_batch([], 10.0, 5).shape == (0, c.N)


def test_served_results_equal_alone_in_the_mix(wmd, setup):
    """Requests arrive while others run (continuous batching over 3 slots);
    each result equals the query run alone, bit for bit."""
    vecs, c, corpus, queries = setup
    alone = _alone(corpus, queries, 10.0, 15, wmd.PREC_FP32)
    srv = wmd.Server(corpus, max_batch=5, slots=3)
    try:
        order = list(range(len(queries))) * 3
        np.random.default_rng(3).shuffle(order)
        tickets = []
        for k, i in enumerate(order):
            tickets.append((i, srv.submit(queries[i][0], queries[i][1], 10.0, 15)))
            if k % 7 == 0:
                time.sleep(0.002)  # let some batches start while more arrive
        for i, t in tickets:
            got = srv.poll(t, timeout_us=30_000_000)
            assert np.array_equal(got, alone[i]), i
        st = srv.stats()
        assert st["completed"] == len(order)
        assert st["batches"] >= len(order) // 5
        assert st["max_batch_seen"] <= 5
    finally:
        srv.close()


def test_server_fault_paths(wmd, setup):
    vecs, c, corpus, queries = setup
    # admission by memory: a budget below one request's need is refused at submit
    need = 2 * corpus.U * 256 * 4
    srv = wmd.Server(corpus, max_batch=4, slots=2, mem_budget=2 * (need // 2), max_pending=4)
    try:
        big = queries[15]  # v_r = 256
        with pytest.raises(wmd.WMDError) as e:
            srv.submit(big[0], big[1], 10.0, 15)
        assert e.value.status == wmd.WMD_ERR_OUT_OF_MEMORY
        # malformed requests never enter the queue
        with pytest.raises(wmd.WMDError) as e:
            srv.submit([1, 1], [0.5, 0.5], 10.0, 15)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
        with pytest.raises(wmd.WMDError) as e:
            srv.submit([1], [1.0], 0.0, 15)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
        # unknown ticket
        with pytest.raises(wmd.WMDError) as e:
            srv.poll(123456789)
        assert e.value.status == wmd.WMD_ERR_INVALID_ARG
        # a flood: the queue holds max_pending requests, then submit refuses
        tickets, refused = [], 0
        for k in range(200):
            q = queries[k % 10]
            try:
                tickets.append((k % 10, srv.submit(q[0], q[1], 10.0, 15)))
            except wmd.WMDError as err:
                assert err.status == wmd.WMD_ERR_NOT_READY
                refused += 1
        assert refused > 0 and tickets
        # a cancelled ticket is gone
        i0, t0 = tickets.pop(0)
        srv.cancel(t0)
        with pytest.raises(wmd.WMDError):
            srv.poll(t0)
        # non-blocking poll answers NOT_READY or the result; bounded poll finishes
        alone = _alone(corpus, queries[:10], 10.0, 15, wmd.PREC_FP32)
        for i, t in tickets:
            try:
                got = srv.poll(t, timeout_us=0)
            except wmd.WMDError as err:
                assert err.status == wmd.WMD_ERR_NOT_READY
                got = srv.poll(t, timeout_us=30_000_000)
            assert np.array_equal(got, alone[i])
    finally:
        srv.close()


def test_server_shutdown_fails_waiting_requests(wmd, setup):
    vecs, c, corpus, queries = setup
    srv = wmd.Server(corpus, max_batch=1, slots=1)
    tickets = [srv.submit(q[0], q[1], 10.0, 15) for q in queries[:8]]
    lib = wmd.lib()
    # destroy while requests wait: none hangs, waiting ones are failed
    srv.close()
    assert srv._h is None
