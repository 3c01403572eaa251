"""Document sharding of a corpus (C ABI ``wmd_shard_plan`` and
``wmd_corpus_load_shard``) and the exchange step that puts the shards'
results together.

The paper splits the documents (the columns of c) into ranges of about equal
nonzeros, one per thread and across sockets (Sec. 3 and 4).  Each column of
x, u and v depends only on its own column of c, so the shards need nothing
from each other until the end: the only exchange is the concatenation of the
shards' WMD slices, or the merge of their k nearest documents.  Everything
here is argument marshalling and that exchange; every distance and every
selection runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import wmd


def plan(row_ptr, doc_idx, V: int, N: int, S: int) -> np.ndarray:
    """``wmd_shard_plan``: boundaries doc_begin[S + 1] of S contiguous
    document ranges with about nnz / S nonzeros each."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    di = np.ascontiguousarray(doc_idx, dtype=np.int32)
    out = np.zeros(int(S) + 1, np.int64)
    wmd._check(wmd.lib().wmd_shard_plan(wmd._ptr(rp), wmd._ptr(di), int(V), int(N), int(S),
                                        wmd._ptr(out)))
    return out


def load_shard(vecs, row_ptr, doc_idx, val, N: int, doc_begin: int, doc_end: int,
               device: int = 0, **opts) -> "wmd.Corpus":
    """``wmd_corpus_load_shard``: a corpus of documents [doc_begin, doc_end)."""
    vecs = np.ascontiguousarray(vecs, dtype=np.float32)
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    di = np.ascontiguousarray(doc_idx, dtype=np.int32)
    vv = np.ascontiguousarray(val, dtype=np.float32)
    V, d = vecs.shape
    o = wmd.options(device=device, **opts)
    h = C.c_void_p()
    wmd._check(wmd.lib().wmd_corpus_load_shard(
        wmd._ptr(vecs), V, d, wmd._ptr(rp), wmd._ptr(di), wmd._ptr(vv), int(N), int(vv.size),
        int(doc_begin), int(doc_end), C.byref(o), C.byref(h)))
    return wmd.Corpus._from_handle(h)


class ShardedCorpus:
    """S document shards of one corpus, each resident on its own device (or
    several on one device).  ``query`` concatenates the shards' WMD slices;
    ``query_topk`` merges their k nearest documents."""

    def __init__(self, vecs, corpus, S: int, devices=None, **opts):
        self.N = corpus.N
        self.bounds = plan(corpus.row_ptr, corpus.doc_idx, corpus.V, corpus.N, S)
        devices = list(devices) if devices is not None else [0] * S
        if len(devices) != S:
            raise ValueError("one device per shard")
        self.shards = [load_shard(vecs, corpus.row_ptr, corpus.doc_idx, corpus.val, corpus.N,
                                  int(self.bounds[s]), int(self.bounds[s + 1]), devices[s], **opts)
                       for s in range(S)]

    def set_loop_variant(self, v_r: int, variant: int, prec: int = wmd.PREC_FP32):
        for sh in self.shards:
            sh.set_loop_variant(v_r, variant, prec)

    def query(self, q_ids, q_w, lam: float, max_iter: int, prec: int = wmd.PREC_FP32):
        """WMD[N]: every shard's slice (``wmd_query``), concatenated."""
        return np.concatenate([sh.query(q_ids, q_w, lam, max_iter, prec) if sh.N else
                               np.zeros(0, np.float64) for sh in self.shards])

    def query_topk(self, q_ids, q_w, lam: float, max_iter: int, k: int,
                   prec: int = wmd.PREC_FP32):
        """The k nearest documents of the whole corpus: each shard's own k
        nearest (``wmd_query_device_topk``), then ``wmd_topk`` over the
        candidates concatenated in shard order.  Returns (ids, values)."""
        import torch
        cand_v, cand_i = [], []
        for s, sh in enumerate(self.shards):
            ks = min(k, sh.N)
            if ks == 0:
                continue
            dq = wmd.DeviceQuery(sh, q_ids, q_w, prec)
            idx = torch.empty(ks, dtype=torch.int64, device=dq.out.device)
            val = torch.empty(ks, dtype=torch.float64, device=dq.out.device)
            sh.query_device_topk(dq.ids, dq.w, dq.v_r, lam, max_iter, prec, dq.ws, dq.ws_bytes,
                                 dq.out, ks, idx, val)
            cand_v.append(val.to(self.shards[0].device))
            cand_i.append(idx.to(self.shards[0].device) + int(self.bounds[s]))
        return merge_candidates(torch.cat(cand_v), torch.cat(cand_i), k)

    def close(self):
        for sh in self.shards:
            sh.close()


def merge_candidates(vals, ids, k: int):
    """The k smallest of the candidates ``vals`` (a device tensor) with their
    document ids ``ids``: ``wmd_topk`` over the values in the order given
    (shard order, which is ascending document order between equal values).
    Returns (ids, values) as numpy arrays."""
    import torch
    k = min(int(k), int(vals.numel()))
    pos = torch.empty(k, dtype=torch.int64, device=vals.device)
    out = torch.empty(k, dtype=torch.float64, device=vals.device)
    if k:
        wmd.topk(vals.contiguous(), int(vals.numel()), k, pos, out)
    return ids[pos].cpu().numpy(), out.cpu().numpy()


# -------------------------------------------------------------- exchange across ranks
def gather_slices(local, counts, group=None):
    """All ranks' WMD slices (1-D float64 tensors of ``counts[r]`` values, on
    the device the process group uses), concatenated in rank order on every
    rank: one all_gather of slices padded to the longest."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    m = max(int(c) for c in counts)
    buf = torch.full((m,), float("nan"), dtype=local.dtype, device=local.device)
    buf[: local.numel()] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([parts[r][: int(counts[r])] for r in range(world)])


def gather_candidates(vals, ids, doc_begin: int, k: int, group=None):
    """All ranks' k-nearest candidates (values and shard-local ids, at most k
    each), with ids shifted to corpus ids, concatenated in rank order:
    (values, ids) tensors on every rank, ready for ``merge_candidates``."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([vals.numel()], dtype=torch.int64, device=vals.device)
    ns = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    pv = torch.full((k,), float("nan"), dtype=torch.float64, device=vals.device)
    pi = torch.full((k,), -1, dtype=torch.int64, device=vals.device)
    pv[: vals.numel()] = vals
    pi[: ids.numel()] = ids + int(doc_begin)
    gv = [torch.empty_like(pv) for _ in range(world)]
    gi = [torch.empty_like(pi) for _ in range(world)]
    dist.all_gather(gv, pv, group=group)
    dist.all_gather(gi, pi, group=group)
    keep = [int(x.item()) for x in ns]
    return (torch.cat([gv[r][: keep[r]] for r in range(world)]),
            torch.cat([gi[r][: keep[r]] for r in range(world)]))
