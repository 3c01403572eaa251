"""Document-sharded corpora on one GPU: S shards (nnz-balanced, as the
paper splits documents across threads and sockets) give exactly the
unsharded corpus's results, slice by slice, and the merged k nearest
documents equal the unsharded selection."""
import numpy as np
import pytest

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2005_06727_gb300 import build as build_mod
    build_mod.build()
    from paper_2005_06727_gb300 import shard, wmd
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return wmd, shard


@pytest.fixture(scope="module")
def data():
    V = 20000
    vecs = synth.make_vecs(V, 96, 41)
    c = synth.make_corpus(V, 1500, 20, 150, 42)
    qs = [synth.make_query(V, n, 43 + n) for n in (7, 30, 100, 200)]
    return vecs, c, qs


@pytest.mark.parametrize("prec_name", ["fp32", "bf16"])
def test_shards_equal_the_unsharded_corpus(mods, data, prec_name):
    wmd, shard = mods
    vecs, c, qs = data
    prec = wmd.PREC_FP32 if prec_name == "fp32" else wmd.PREC_BF16_K
    whole = wmd.Corpus.from_synth(vecs, c)
    for q in qs:
        whole.set_loop_variant(len(q[0]), 0, prec)
    want = [whole.query(q[0], q[1], 10.0, 15, prec) for q in qs]
    whole.close()
    for S in (2, 3):
        sc = shard.ShardedCorpus(vecs, c, S)
        assert [sh.N for sh in sc.shards] == list(np.diff(sc.bounds))
        for q, w in zip(qs, want):
            sc.set_loop_variant(len(q[0]), 0, prec)
            np.testing.assert_array_equal(sc.query(q[0], q[1], 10.0, 15, prec), w)
        sc.close()


def test_sharded_k_nearest_equal_the_unsharded_selection(mods, data):
    import torch
    wmd, shard = mods
    vecs, c, qs = data
    whole = wmd.Corpus.from_synth(vecs, c)
    sc = shard.ShardedCorpus(vecs, c, 3)
    for q in qs[1:3]:
        whole.set_loop_variant(len(q[0]), 0)
        sc.set_loop_variant(len(q[0]), 0)
        full = whole.query(q[0], q[1], 10.0, 15)
        for k in (1, 10, 200):
            d = torch.from_numpy(full).cuda()
            idx = torch.empty(k, dtype=torch.int64, device="cuda")
            val = torch.empty(k, dtype=torch.float64, device="cuda")
            wmd.topk(d, c.N, k, idx, val)
            ids, vals = sc.query_topk(q[0], q[1], 10.0, 15, k)
            np.testing.assert_array_equal(ids, idx.cpu().numpy())
            np.testing.assert_array_equal(vals, val.cpu().numpy())
            # and the oracle's rule on the full vector
            oi, ov = orc.nearest_documents(full, k)
            np.testing.assert_array_equal(ids, oi)
    # against the FP64 oracle on a few documents of one shard boundary
    q = qs[1]
    b = int(sc.bounds[1])
    docs = np.arange(max(0, b - 20), min(c.N, b + 20))
    want = orc.sinkhorn_wmd_sparse(q[0], q[1], c.row_ptr, c.doc_idx, c.val, c.N, vecs, 10.0, 15,
                                   docs=docs)
    got = sc.query(q[0], q[1], 10.0, 15)[docs]
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-5
    sc.close()
    whole.close()
