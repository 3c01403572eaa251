"""Document sharding on the host: the nnz-balanced plan (C ABI, no GPU) and
the exchange step across ranks (two gloo processes on the CPU), checked
against the oracle's selection rule for the k nearest documents."""
import os
import socket

import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import shard, synth, wmd


def test_plan_is_contiguous_and_balanced():
    c = synth.make_corpus(3000, 500, 5, 90, 17)
    lens = np.diff(c.doc_ptr)
    for S in (1, 2, 3, 7, 16):
        b = shard.plan(c.row_ptr, c.doc_idx, c.V, c.N, S)
        assert b[0] == 0 and b[-1] == c.N and np.all(np.diff(b) >= 0)
        per = np.array([lens[b[s]:b[s + 1]].sum() for s in range(S)])
        assert per.sum() == c.nnz
        # every shard within one document of the ideal nnz / S
        assert np.abs(per - c.nnz / S).max() <= lens.max()


def test_plan_edge_cases_and_errors():
    c = synth.make_corpus(200, 3, 2, 5, 1)
    b = shard.plan(c.row_ptr, c.doc_idx, c.V, c.N, 8)      # more shards than documents
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)
    empty = synth.corpus_from_docs(50, [])
    assert list(shard.plan(empty.row_ptr, empty.doc_idx, 50, 0, 2)) == [0, 0, 0]
    with pytest.raises(wmd.WMDError):
        shard.plan(c.row_ptr, c.doc_idx, c.V, c.N, 0)
    bad = c.doc_idx.copy()
    bad[0] = 99
    with pytest.raises(wmd.WMDError):
        shard.plan(c.row_ptr, bad, c.V, c.N, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, bounds, full, k, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = int(bounds[rank]), int(bounds[rank + 1])
        local = torch.from_numpy(full[lo:hi].copy())
        counts = np.diff(bounds)
        got = shard.gather_slices(local, counts)
        # each rank's own k nearest by the oracle's rule, then the exchange
        ids, vals = orc.nearest_documents(full[lo:hi], min(k, hi - lo))
        cv, ci = shard.gather_candidates(torch.from_numpy(vals), torch.from_numpy(ids), lo, k)
        q.put((rank, got.numpy(), cv.numpy(), ci.numpy()))
    finally:
        dist.destroy_process_group()


def test_exchange_across_two_gloo_ranks():
    import multiprocessing as mp
    rng = np.random.default_rng(5)
    full = rng.uniform(1.0, 2.0, 37)
    full[[3, 20]] = full[11]          # ties across the two shards
    full[30] = np.nan                 # an empty document
    bounds = np.array([0, 15, 37])
    k = 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, bounds, full, k, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_ids, want_vals = orc.nearest_documents(full, k)
    for _, got, cv, ci in out:
        np.testing.assert_array_equal(got, full)
        # the candidates in shard order hold the global answer; the oracle's
        # rule over them (position order = document order) picks it
        sel, _ = orc.nearest_documents(cv, k)
        np.testing.assert_array_equal(ci[sel], want_ids)
        np.testing.assert_array_equal(cv[sel], want_vals)
