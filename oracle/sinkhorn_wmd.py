"""Plain FP64 CPU oracle for the sparse one-query-versus-many-documents
Sinkhorn-Knopp Word Mover's Distance (Tithi & Petrini, arXiv 2005.06727).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously correct
statement of what the CUDA path must compute.  Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  It shares no code with the CUDA library and never imports it.

Every step follows the paper, in its order and notation:

* Sec. 2 defines the word-to-word cost as the unsquared Euclidean distance
  m(i, j) = sqrt(sum_k (e_i[k] - e_j[k])^2) between embedding rows.
* Algorithm 1 (Sec. 3, after Cuturi 2013):
    I = (r > 0); r = r(I); M = M(I, :); K = exp(-lambda M)
    x = ones(length(r), size(c, 2)) / length(r)
    repeat: x = diag(1./r) K (c .* (1 ./ (K^T (1./x))))
    u = 1./x;  v = c .* (1 ./ (K^T u))
    d = sum(u .* ((K .* M) v))            (a sum over the query rows)
* Sec. 3 ("A Python Implementation", Table 1) fixes the loop as exactly
  ``max_iter`` bodies ``u = 1/x; v = c.multiply(1/(K^T u)); x = K_over_r v``
  followed by one more ``u``/``v`` update and the reduction, i.e. max_iter+1
  SDDMMs and max_iter SpMMs.  ``max_iter = 0`` is allowed.
* Sec. 3 ("Dense to Sparse Kernel") evaluates K^T u only at the nonzeros of c
  (SDDMM) and forms x with a dense-times-sparse product (SpMM).

Readings where the paper is silent or ambiguous:
m(i, j) is unsquared (the sqrt formula of Sec. 2 wins over the "||.||^2"
notation); lambda is passed positive and K = exp(-lambda M) (Algorithm 1; the
paper's Python negates lambda before the call); r and c are used as given, no
renormalisation; IEEE arithmetic decides empty documents (NaN for
max_iter >= 1, because u = 1/0 meets a zero column of (K.*M) v).

Inputs are float32 arrays (the format the library takes); the oracle widens
them to float64 and computes everything in float64.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# Algorithm 1, query selection: I = (r > 0)
# --------------------------------------------------------------------------
def select_nonzero(q_ids, q_w):
    """Keep the query words with positive weight (Algorithm 1: I = (r > 0)).

    Returns (ids int64 [v_r], r float64 [v_r]) in the given order.
    """
    ids = np.asarray(q_ids, dtype=np.int64)
    w = np.asarray(q_w, dtype=np.float32).astype(np.float64)
    keep = w > 0
    return ids[keep], w[keep]


# --------------------------------------------------------------------------
# Sec. 2: m(i, j) = sqrt(sum((embedding[i] - embedding[j])^2))
# --------------------------------------------------------------------------
def cdist(vecs, rows_a, rows_b, chunk: int = 2048):
    """Euclidean distances between embedding rows, direct-difference form.

    M[a, b] = sqrt(sum_k (vecs[rows_a[a], k] - vecs[rows_b[b], k])^2), in float64
    from the float32 table widened to float64 (Sec. 2).
    """
    A = np.asarray(vecs[np.asarray(rows_a, dtype=np.int64)], dtype=np.float64)
    rows_b = np.asarray(rows_b, dtype=np.int64)
    out = np.empty((A.shape[0], rows_b.shape[0]), dtype=np.float64)
    for s in range(0, rows_b.shape[0], chunk):
        B = np.asarray(vecs[rows_b[s:s + chunk]], dtype=np.float64)
        diff = A[:, None, :] - B[None, :, :]
        out[:, s:s + chunk] = np.sqrt(np.sum(diff * diff, axis=2))
    return out


# --------------------------------------------------------------------------
# Algorithm 1, dense (Cuturi) form -- tiny inputs only
# --------------------------------------------------------------------------
def sinkhorn_wmd_dense(r, c, vecs, lam, max_iter, return_state=False):
    """Algorithm 1 written out with dense matrices.

    r: dense query histogram, shape [V]; c: dense V x N target histograms;
    vecs: V x d embeddings.  Returns WMD[N] (and u, v, K, M, r_I if asked).
    """
    r = np.asarray(r, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    E = np.asarray(vecs, dtype=np.float64)
    I = r > 0                                    # I = (r > 0)
    r_I = r[I]                                   # r = r(I)
    diff = E[I][:, None, :] - E[None, :, :]      # M = M(I, :), Sec. 2 distance
    M = np.sqrt(np.sum(diff * diff, axis=2))
    K = np.exp(-lam * M)                         # K = exp(-lambda M)
    v_r = r_I.shape[0]
    x = np.ones((v_r, c.shape[1])) / v_r         # x = ones(length(r), size(c,2))/length(r)
    with np.errstate(divide="ignore", invalid="ignore"):
        for _ in range(max_iter):                # "while x changes" -> max_iter bodies
            x = np.diag(1.0 / r_I) @ K @ (c * (1.0 / (K.T @ (1.0 / x))))
        u = 1.0 / x
        v = c * (1.0 / (K.T @ u))
        wmd = np.sum(u * ((K * M) @ v), axis=0)
    if return_state:
        return wmd, dict(u=u, v=v, K=K, M=M, r=r_I)
    return wmd


# --------------------------------------------------------------------------
# Sec. 3 sparse form: SDDMM at the nonzeros of c, then SpMM
# --------------------------------------------------------------------------
def sinkhorn_wmd_sparse(q_ids, q_w, row_ptr, doc_idx, val, N, vecs, lam, max_iter,
                        docs=None, return_state=False):
    """The paper's sparse formulation of Algorithm 1.

    c is given in the paper's layout, a V x N CSR matrix with rows = words
    (``row_ptr`` [V+1], ``doc_idx`` [nnz], ``val`` [nnz]).  Per loop body:

      u = 1/x
      SDDMM:  s_wj = sum_i K[i, w] u[i, j]   for every nonzero (w, j) of c
              v_wj = c_wj / s_wj
      SpMM:   x = diag(1/r) (K v)            (v sparse with c's pattern)

    then u = 1/x, one more SDDMM for v, and WMD_j = sum_i u_ij ((K.*M) v)_ij.

    ``docs`` optionally restricts the computation to a subset of the columns of
    c (every column of x, u and v depends only on the same column of c, so a
    subset gives the same values for those documents).  Only the vocabulary
    words that occur in the selected documents need a column of M.
    """
    ids, r = select_nonzero(q_ids, q_w)
    v_r = ids.shape[0]
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    V = row_ptr.shape[0] - 1
    w_nz = np.repeat(np.arange(V, dtype=np.int64), np.diff(row_ptr))
    j_nz = np.asarray(doc_idx, dtype=np.int64)
    c_nz = np.asarray(val, dtype=np.float32).astype(np.float64)
    if docs is not None:
        docs = np.asarray(docs, dtype=np.int64)
        pos = np.full(N, -1, dtype=np.int64)
        pos[docs] = np.arange(docs.shape[0])
        keep = pos[j_nz] >= 0
        w_nz, j_nz, c_nz = w_nz[keep], pos[j_nz[keep]], c_nz[keep]
        N = docs.shape[0]

    words = np.unique(w_nz)                      # vocabulary columns touched by c
    col = np.searchsorted(words, w_nz)           # nonzero -> column of M / K
    M = cdist(vecs, ids, words)                  # v_r x |words|
    K = np.exp(-lam * M)
    KM = K * M
    K_nz = K[:, col]                             # K[:, w] for every nonzero

    def spmm(A, v):
        """A (v_r x |words|) times the sparse matrix v with c's pattern."""
        vs = sp.csr_matrix((v, (j_nz, col)), shape=(N, words.shape[0]))
        return np.asarray((vs @ A.T).T)

    x = np.ones((v_r, N)) / v_r
    with np.errstate(divide="ignore", invalid="ignore"):
        for _ in range(max_iter):
            u = 1.0 / x
            s = np.sum(K_nz * u[:, j_nz], axis=0)   # SDDMM
            v = c_nz / s
            x = (1.0 / r)[:, None] * spmm(K, v)      # SpMM with K_over_r
        u = 1.0 / x
        s = np.sum(K_nz * u[:, j_nz], axis=0)
        v = c_nz / s
        wmd = np.sum(u * spmm(KM, v), axis=0)
    if return_state:
        return wmd, dict(u=u, v_nz=v, w_nz=w_nz, j_nz=j_nz, K=K, M=M, words=words, r=r)
    return wmd


# --------------------------------------------------------------------------
# Algorithm 1's stopping rule "while x changes", per document
# --------------------------------------------------------------------------
def sinkhorn_wmd_sparse_until_converged(q_ids, q_w, row_ptr, doc_idx, val, N, vecs, lam,
                                        max_iter, tol, iters=None, docs=None):
    """The sparse form of Algorithm 1 with its loop condition "while x changes".

    Algorithm 1 repeats its body while x changes; Sec. 3 caps the loop at
    ``max_iter`` bodies.  Every column j of x depends only on column j of c, so
    the test is taken per document: after body k (k = 1, 2, ...) has produced
    x^(k), document j stops iterating when x no longer changes by more than
    ``tol`` relative to its previous value,

        rho_j^(k) = max_i |x^(k)_ij - x^(k-1)_ij| / x^(k-1)_ij  <=  tol,

    or when k = max_iter.  Its result is then taken as after exactly T_j = k
    bodies: u = 1/x^(k), one more SDDMM for v, and the WMD reduction.  A
    stopped document's x is frozen while the others go on.  NaN never passes
    the test, so an empty document (x^(1) = 0, then 0/0) runs max_iter bodies.
    ``tol`` is taken in [0, 1).

    ``iters`` (optional, int [N]) replaces the rule: document j then runs
    exactly iters[j] bodies (0 <= iters[j] <= max_iter).  ``docs`` restricts
    the computation to a subset of the documents, as in sinkhorn_wmd_sparse.

    Returns (wmd [N], T [N] int, rho [max_iter, N]) where rho[k-1, j] is
    rho_j^(k) while document j was still running and NaN afterwards.
    """
    if not 0.0 <= tol < 1.0:
        raise ValueError("tol must lie in [0, 1)")
    ids, r = select_nonzero(q_ids, q_w)
    v_r = ids.shape[0]
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    V = row_ptr.shape[0] - 1
    w_nz = np.repeat(np.arange(V, dtype=np.int64), np.diff(row_ptr))
    j_nz = np.asarray(doc_idx, dtype=np.int64)
    c_nz = np.asarray(val, dtype=np.float32).astype(np.float64)
    if docs is not None:
        docs = np.asarray(docs, dtype=np.int64)
        pos = np.full(N, -1, dtype=np.int64)
        pos[docs] = np.arange(docs.shape[0])
        keep = pos[j_nz] >= 0
        w_nz, j_nz, c_nz = w_nz[keep], pos[j_nz[keep]], c_nz[keep]
        N = docs.shape[0]
        if iters is not None:
            iters = np.asarray(iters)[docs]

    words = np.unique(w_nz)
    col = np.searchsorted(words, w_nz)
    M = cdist(vecs, ids, words)
    K = np.exp(-lam * M)
    KM = K * M
    K_nz = K[:, col]

    def spmm(A, v):
        vs = sp.csr_matrix((v, (j_nz, col)), shape=(N, words.shape[0]))
        return np.asarray((vs @ A.T).T)

    x = np.ones((v_r, N)) / v_r
    T = np.zeros(N, dtype=np.int64)
    running = np.ones(N, dtype=bool) if iters is None else np.asarray(iters) > 0
    rho = np.full((max(max_iter, 0), N), np.nan)
    with np.errstate(divide="ignore", invalid="ignore"):
        for k in range(1, max_iter + 1):
            if not running.any():
                break
            u = 1.0 / x
            s = np.sum(K_nz * u[:, j_nz], axis=0)       # SDDMM
            v = c_nz / s
            x_new = (1.0 / r)[:, None] * spmm(K, v)     # SpMM with K_over_r
            change = np.max(np.abs(x_new - x) / x, axis=0) if v_r else np.zeros(N)
            rho[k - 1, running] = change[running]
            x[:, running] = x_new[:, running]           # stopped documents keep their x
            T[running] = k
            if iters is None:
                running &= ~(change <= tol)             # "while x changes"
                if k == max_iter:
                    running[:] = False
            else:
                running &= np.asarray(iters) > k
        u = 1.0 / x
        s = np.sum(K_nz * u[:, j_nz], axis=0)
        v = c_nz / s
        wmd = np.sum(u * spmm(KM, v), axis=0)
    return wmd, T, rho


# --------------------------------------------------------------------------
# k nearest documents (the retrieval use of the WMD, Sec. 1 and 2)
# --------------------------------------------------------------------------
def nearest_documents(wmd, k):
    """The k documents with the smallest WMD, nearest first.

    Ordering: by value (-0 equals +0), ties by the lower document id, and
    every NaN (an empty document) after every number, so the answer is unique.
    Returns (ids int64 [k], values float64 [k]).
    """
    w = np.asarray(wmd, dtype=np.float64)
    order = sorted(range(w.shape[0]),
                   key=lambda j: (bool(np.isnan(w[j])), 0.0 if np.isnan(w[j]) else float(w[j]), j))
    ids = np.array(order[:k], dtype=np.int64)
    return ids, w[ids]


# --------------------------------------------------------------------------
# Exact EMD for tiny equal-size uniform histograms (used to pin the oracle)
# --------------------------------------------------------------------------
def emd_uniform_bruteforce(M):
    """Exact optimal transport cost between two uniform n-point histograms.

    With both marginals equal to 1/n the transport polytope is the Birkhoff
    polytope scaled by 1/n, whose vertices are permutation matrices, so the
    optimum is min over permutations pi of (1/n) sum_i M[i, pi(i)].
    """
    import itertools
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    best = np.inf
    for perm in itertools.permutations(range(n)):
        best = min(best, M[np.arange(n), perm].sum())
    return best / n
