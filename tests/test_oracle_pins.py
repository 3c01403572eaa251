"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests compare the oracle with itself under another name: each
one checks a closed form, an invariant, an independent library routine or a
brute-force solution.  A dropped term, a wrong sign, a transposed operand or a
squared distance in the oracle fails at least one of them (see
``test_planted_mistakes_are_caught``).
"""
import itertools

import numpy as np
import pytest
import scipy.optimize
import scipy.spatial.distance

from oracle import sinkhorn_wmd as orc
from paper_2005_06727_gb300 import synth


def _small_problem(V=60, d=16, N=7, lo=2, hi=9, vr=5, seed=0):
    vecs = synth.make_vecs(V, d, seed + 11)
    corpus = synth.make_corpus(V, N, lo, hi, seed + 12)
    q_ids, q_w = synth.make_query(V, vr, seed + 13)
    return vecs, corpus, q_ids, q_w


def _sparse(vecs, c, q_ids, q_w, lam, T, **kw):
    return orc.sinkhorn_wmd_sparse(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N,
                                   vecs, lam, T, **kw)


def _one_doc_corpus(V, words, weights):
    return synth.corpus_from_docs(V, [(np.asarray(words, np.int32), np.asarray(weights, np.float32))])


# ---------------------------------------------------------------- P7: cdist
def test_cdist_matches_scipy_and_is_exact_on_identical_rows():
    """Sec. 2 distance against SciPy's cdist (an independent implementation)."""
    vecs = synth.make_vecs(300, 300, 5)
    a = np.array([0, 7, 299, 42])
    b = np.arange(300)
    ours = orc.cdist(vecs, a, b, chunk=64)
    ref = scipy.spatial.distance.cdist(vecs[a].astype(np.float64), vecs.astype(np.float64))
    np.testing.assert_allclose(ours, ref, rtol=1e-13, atol=1e-15)
    # identical vocabulary rows are exactly zero apart
    for k, w in enumerate(a):
        assert ours[k, w] == 0.0
    # unsquared reading: distance between N(0,1/d) rows is about sqrt(2), not 2
    assert 1.2 < np.median(ours) < 1.6


# ---------------------------------------------------------------- P1: dense == sparse
@pytest.mark.parametrize("T", [0, 1, 3, 15])
def test_dense_equals_sparse_small(T):
    """The sparse SDDMM/SpMM form equals the dense Algorithm 1 (Sec. 3)."""
    vecs, c, q_ids, q_w = _small_problem()
    r = synth.dense_r(c.V, q_ids, q_w)
    dense = orc.sinkhorn_wmd_dense(r, synth.dense_c(c), vecs, 10.0, T)
    sparse = _sparse(vecs, c, q_ids, q_w, 10.0, T)
    np.testing.assert_allclose(sparse, dense, rtol=1e-12)


def test_dense_equals_sparse_tiny_workload():
    """Same identity on the tiny workload (V=2000, N=100, v_r=20, lambda=10, T=15)."""
    w = synth.TINY
    vecs, c, queries = synth.make_workload(w)
    q_ids, q_w = queries[0]
    r = synth.dense_r(w.V, q_ids, q_w)
    dense = orc.sinkhorn_wmd_dense(r, synth.dense_c(c), vecs, w.lam, w.max_iter)
    sparse = _sparse(vecs, c, q_ids, q_w, w.lam, w.max_iter)
    assert np.all(np.isfinite(sparse))
    np.testing.assert_allclose(sparse, dense, rtol=1e-12)
    # a subset of the documents gives the same values for those documents
    docs = np.array([3, 50, 99, 0])
    sub = _sparse(vecs, c, q_ids, q_w, w.lam, w.max_iter, docs=docs)
    np.testing.assert_allclose(sub, sparse[docs], rtol=1e-13)


# ---------------------------------------------------------------- P2: v_r = 1
@pytest.mark.parametrize("T", [0, 1, 7])
@pytest.mark.parametrize("lam", [1.0, 10.0])
def test_single_query_word_closed_form(T, lam):
    """With one query word the only feasible plan ships all mass from it:
    WMD_j = sum_w c_wj m(q, w), for every lambda and every T."""
    vecs, c, _, _ = _small_problem()
    q_ids = np.array([17], np.int32)
    q_w = np.array([1.0], np.float32)
    got = _sparse(vecs, c, q_ids, q_w, lam, T)
    M = scipy.spatial.distance.cdist(vecs[[17]].astype(np.float64), vecs.astype(np.float64))[0]
    want = np.array([np.sum(c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]].astype(np.float64)
                            * M[c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]]]) for j in range(c.N)])
    np.testing.assert_allclose(got, want, rtol=1e-12)


# ---------------------------------------------------------------- P3: one-word doc
@pytest.mark.parametrize("T", [1, 2, 15])
def test_single_word_document_closed_form(T):
    """A target with one word w (weight c) receives all mass:
    WMD = c * sum_i r_i m(i, w) / sum_i r_i, for T >= 1."""
    vecs, _, q_ids, q_w = _small_problem()
    V = vecs.shape[0]
    for w_word, cw in [(3, 1.0), (int(q_ids[0]), 1.0), (41, 0.625)]:
        c = _one_doc_corpus(V, [w_word], [cw])
        got = _sparse(vecs, c, q_ids, q_w, 10.0, T)[0]
        r = q_w.astype(np.float64)
        M = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64),
                                         vecs[[w_word]].astype(np.float64))[:, 0]
        want = np.float64(np.float32(cw)) * np.sum(r * M) / np.sum(r)
        np.testing.assert_allclose(got, want, rtol=1e-12)


# ---------------------------------------------------------------- P4: T = 0
def test_zero_iterations_closed_form():
    """With x = 1/v_r, u is constant and WMD_j = sum_w c_wj (sum_i K_iw M_iw)/(sum_i K_iw)."""
    vecs, c, q_ids, q_w = _small_problem()
    lam = 3.0
    got = _sparse(vecs, c, q_ids, q_w, lam, 0)
    M = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64), vecs.astype(np.float64))
    K = np.exp(-lam * M)
    per_word = (K * M).sum(0) / K.sum(0)
    want = np.array([np.sum(c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]].astype(np.float64)
                            * per_word[c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]]]) for j in range(c.N)])
    np.testing.assert_allclose(got, want, rtol=1e-12)


# ---------------------------------------------------------------- P5: marginals
def test_marginals():
    """P = diag(u) K diag(v) (Eq. 1): its columns equal c after the final v
    update, and its rows approach r as the iteration count grows."""
    vecs, c, q_ids, q_w = _small_problem(N=4, lo=4, hi=8, vr=4, seed=3)
    r = synth.dense_r(c.V, q_ids, q_w)
    cd = synth.dense_c(c)
    errs = []
    for T in [1, 4, 16, 64, 400]:
        _, st = orc.sinkhorn_wmd_dense(r, cd, vecs, 4.0, T, return_state=True)
        for j in range(c.N):
            P = st["u"][:, j][:, None] * st["K"] * st["v"][:, j][None, :]
            np.testing.assert_allclose(P.sum(0), cd[:, j], rtol=1e-12, atol=1e-15)
        row_err = max(np.abs((st["u"][:, j][:, None] * st["K"] * st["v"][:, j][None, :]).sum(1)
                             - st["r"] / st["r"].sum() * cd[:, j].sum()).sum() for j in range(c.N))
        errs.append(row_err)
    assert all(b <= a * (1 + 1e-9) for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-10


# ---------------------------------------------------------------- 2 x 2 closed form
def test_two_by_two_closed_form():
    """For a 2x2 plan with margins r, c the fixed point of Sinkhorn-Knopp has
    P11 P22 / (P12 P21) = K11 K22 / (K12 K21); with P12 = r1 - p, P21 = c1 - p,
    P22 = 1 - r1 - c1 + p this is a quadratic in p = P11."""
    V, d = 6, 8
    vecs = synth.make_vecs(V, d, 99)
    q_ids = np.array([0, 1], np.int32)
    q_w = np.array([0.25, 0.75], np.float32)
    c = _one_doc_corpus(V, [3, 5], [0.625, 0.375])
    lam = 2.5
    got = _sparse(vecs, c, q_ids, q_w, lam, 3000)[0]

    r1 = np.float64(np.float32(0.25))
    c1 = np.float64(np.float32(0.625))
    M = scipy.spatial.distance.cdist(vecs[[0, 1]].astype(np.float64), vecs[[3, 5]].astype(np.float64))
    K = np.exp(-lam * M)
    kappa = K[0, 0] * K[1, 1] / (K[0, 1] * K[1, 0])
    a = 1.0 - kappa
    b = (1.0 - r1 - c1) + kappa * (r1 + c1)
    cc = -kappa * r1 * c1
    roots = np.roots([a, b, cc]).real
    lo, hi = max(0.0, r1 + c1 - 1.0), min(r1, c1)
    p = [t for t in roots if lo - 1e-12 <= t <= hi + 1e-12]
    assert len(p) == 1
    p = p[0]
    P = np.array([[p, r1 - p], [c1 - p, 1.0 - r1 - c1 + p]])
    np.testing.assert_allclose(got, np.sum(P * M), rtol=1e-11)


# ---------------------------------------------------------------- entropic OT dual
def test_converged_value_matches_entropic_dual_solution():
    """At convergence the oracle's WMD is <P*, M> for the unique minimiser P*
    of <P, M> + (1/lambda) sum P (log P - 1) under the marginals r, c (Eq. 1).
    Here P* comes from maximising the smooth dual with L-BFGS instead."""
    V, d = 12, 10
    vecs = synth.make_vecs(V, d, 4)
    q_ids = np.array([0, 2, 4], np.int32)
    # binary fractions: both margins sum to exactly 1 in float32
    q_w = np.array([0.25, 0.5, 0.25], np.float32)
    c = _one_doc_corpus(V, [5, 7, 9, 11], [0.125, 0.375, 0.25, 0.25])
    lam = 3.0
    got = _sparse(vecs, c, q_ids, q_w, lam, 5000)[0]

    r = q_w.astype(np.float64)
    cv = c.doc_vals.astype(np.float64)
    M = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64), vecs[c.doc_words].astype(np.float64))

    def negdual(z):
        f, g = z[:3], z[3:]
        P = np.exp(lam * (f[:, None] + g[None, :] - M))
        val = f @ r + g @ cv - P.sum() / lam
        grad = np.concatenate([r - P.sum(1), cv - P.sum(0)])
        return -val, -grad

    res = scipy.optimize.minimize(negdual, np.zeros(7), jac=True, method="L-BFGS-B",
                                  options=dict(ftol=1e-15, gtol=1e-13, maxiter=10000))
    f, g = res.x[:3], res.x[3:]
    P = np.exp(lam * (f[:, None] + g[None, :] - M))
    np.testing.assert_allclose(P.sum(1), r, atol=1e-9)
    np.testing.assert_allclose(got, np.sum(P * M), rtol=1e-7)


# ---------------------------------------------------------------- P6: >= EMD
def test_emd_bruteforce_matches_assignment_solver():
    rng = np.random.default_rng(0)
    for n in range(1, 7):
        M = rng.random((n, n))
        ri, ci = scipy.optimize.linear_sum_assignment(M)
        assert abs(orc.emd_uniform_bruteforce(M) - M[ri, ci].sum() / n) < 1e-14


@pytest.mark.parametrize("n", [3, 4, 5])
def test_sinkhorn_at_least_emd_and_gap_shrinks(n):
    """The entropic plan is feasible, so its cost is >= the exact EMD; the gap
    closes as lambda grows (the Sinkhorn distance tends to the OT distance)."""
    V, d = 40, 300
    vecs = synth.make_vecs(V, d, 21 + n)
    rng = np.random.default_rng(n)
    words = rng.choice(V, 2 * n, replace=False)
    q_ids = np.sort(words[:n]).astype(np.int32)
    doc = np.sort(words[n:]).astype(np.int32)
    q_w = np.full(n, 1.0 / n, np.float32)
    # equal-size uniform histograms; use exact 1/n weights in float32 for both sides
    c = _one_doc_corpus(V, doc, np.full(n, 1.0 / n, np.float32))
    M = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64), vecs[doc].astype(np.float64))
    emd = orc.emd_uniform_bruteforce(M)
    gaps = []
    for lam in [10.0, 40.0, 160.0]:
        got, st = _sparse(vecs, c, q_ids, q_w, lam, 20000, return_state=True)
        # row marginal error bounds how far the plan is from feasibility
        u = st["u"][:, 0]
        K = st["K"]
        col = np.searchsorted(st["words"], doc)
        P = u[:, None] * K[:, col] * st["v_nz"][None, :]
        slack = M.max() * np.abs(P.sum(1) - q_w.astype(np.float64)).sum()
        assert got[0] >= emd - slack - 1e-12
        gaps.append(got[0] - emd)
    assert gaps[0] > gaps[1] > gaps[2] >= -1e-9
    assert gaps[2] / emd < 0.05


# ---------------------------------------------------------------- P8: invariances
def test_permutation_invariance():
    vecs, c, q_ids, q_w = _small_problem(seed=8)
    base = _sparse(vecs, c, q_ids, q_w, 10.0, 15)
    # permute the documents
    perm = np.random.default_rng(1).permutation(c.N)
    docs = [(c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]], c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]]) for j in perm]
    c2 = synth.corpus_from_docs(c.V, docs)
    np.testing.assert_allclose(_sparse(vecs, c2, q_ids, q_w, 10.0, 15), base[perm], rtol=1e-12)
    # permute the query words
    qp = np.random.default_rng(2).permutation(len(q_ids))
    np.testing.assert_allclose(_sparse(vecs, c, q_ids[qp], q_w[qp], 10.0, 15), base, rtol=1e-12)
    # relabel the vocabulary (embedding rows move with their ids)
    vp = np.random.default_rng(3).permutation(c.V)
    inv = np.argsort(vp)
    vecs2 = vecs[inv]                      # new id vp[w] holds old row w
    docs3 = [(vp[c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]]], c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]]) for j in range(c.N)]
    docs3 = [(ids[np.argsort(ids)].astype(np.int32), w[np.argsort(ids)]) for ids, w in docs3]
    c3 = synth.corpus_from_docs(c.V, docs3)
    np.testing.assert_allclose(_sparse(vecs2, c3, vp[q_ids].astype(np.int32), q_w, 10.0, 15), base, rtol=1e-12)


# ---------------------------------------------------------------- degenerate inputs
def test_empty_document_and_zero_weights():
    vecs, c, q_ids, q_w = _small_problem(seed=9)
    docs = [(c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]], c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]]) for j in range(c.N)]
    docs.insert(2, (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    c2 = synth.corpus_from_docs(c.V, docs)
    r = synth.dense_r(c2.V, q_ids, q_w)
    for T in [0, 1, 15]:
        sp_ = _sparse(vecs, c2, q_ids, q_w, 10.0, T)
        de = orc.sinkhorn_wmd_dense(r, synth.dense_c(c2), vecs, 10.0, T)
        if T == 0:
            assert sp_[2] == 0.0 and de[2] == 0.0
        else:
            assert np.isnan(sp_[2]) and np.isnan(de[2])
        keep = np.arange(c2.N) != 2
        np.testing.assert_allclose(sp_[keep], de[keep], rtol=1e-12)
    # a zero-weight query word is dropped (I = r > 0)
    q_ids2 = np.concatenate([q_ids, [int(c.V - 1)]]).astype(np.int32)
    q_w2 = np.concatenate([q_w, [0.0]]).astype(np.float32)
    np.testing.assert_allclose(_sparse(vecs, c, q_ids2, q_w2, 10.0, 15),
                               _sparse(vecs, c, q_ids, q_w, 10.0, 15), rtol=1e-15)


# ---------------------------------------------------------------- the pins bite
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible mistakes in the oracle (on the CPU) and check that the
    closed-form pins above reject each of them."""
    vecs, c, q_ids, q_w = _small_problem(seed=5)
    M1 = scipy.spatial.distance.cdist(vecs[[17]].astype(np.float64), vecs.astype(np.float64))[0]
    want_vr1 = np.array([np.sum(c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]].astype(np.float64)
                                * M1[c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]]]) for j in range(c.N)])
    real_cdist = orc.cdist

    def squared(vecs_, a, b, chunk=2048):
        return real_cdist(vecs_, a, b, chunk) ** 2

    monkeypatch.setattr(orc, "cdist", squared)
    got = _sparse(vecs, c, np.array([17], np.int32), np.array([1.0], np.float32), 10.0, 5)
    assert not np.allclose(got, want_vr1, rtol=1e-6)
    monkeypatch.setattr(orc, "cdist", real_cdist)

    # dropping the diag(1/r) factor breaks the single-word-document closed form
    src = orc.sinkhorn_wmd_sparse

    def no_r(q_ids_, q_w_, *a, **k):
        ids, r = orc.select_nonzero(q_ids_, q_w_)
        return src(ids, np.ones_like(r, dtype=np.float32) / len(r), *a, **k)

    cw = _one_doc_corpus(vecs.shape[0], [3], [1.0])
    q_w = np.array([0.5, 0.25, 0.125, 0.0625, 0.0625], np.float32)[:len(q_ids)]
    r = q_w.astype(np.float64)
    Mq = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64), vecs[[3]].astype(np.float64))[:, 0]
    want = np.sum(r * Mq) / np.sum(r)
    bad = no_r(q_ids, q_w, cw.row_ptr, cw.doc_idx, cw.val, cw.N, vecs, 10.0, 3)[0]
    assert abs(bad - want) > 1e-6 * want


# ---------------------------------------------------------------- "while x changes"
def _conv(vecs, c, q_ids, q_w, lam, T, tol, **kw):
    return orc.sinkhorn_wmd_sparse_until_converged(q_ids, q_w, c.row_ptr, c.doc_idx, c.val, c.N,
                                                   vecs, lam, T, tol, **kw)


def test_forced_iteration_counts_equal_fixed_iteration_runs():
    """Freezing a document after T_j bodies gives exactly the fixed-count
    result at max_iter = T_j (columns of x are independent, Algorithm 1)."""
    vecs, c, q_ids, q_w = _small_problem(N=12, seed=31)
    T = np.random.default_rng(4).integers(0, 9, c.N)
    T[3] = 0
    wmd, got_T, _ = _conv(vecs, c, q_ids, q_w, 10.0, 8, 0.0, iters=T)
    assert np.array_equal(got_T, T)
    for t in np.unique(T):
        docs = np.flatnonzero(T == t)
        want = _sparse(vecs, c, q_ids, q_w, 10.0, int(t), docs=docs)
        np.testing.assert_allclose(wmd[docs], want, rtol=1e-13)


@pytest.mark.parametrize("tol", [1e-2, 1e-3])
def test_stopping_rule_is_relative_change_of_x(tol):
    """T_j is the first body k after which max_i |x^(k) - x^(k-1)| / x^(k-1)
    <= tol; x^(k) is taken independently from fixed-count runs (x = 1/u)."""
    vecs, c, q_ids, q_w = _small_problem(V=80, N=9, lo=3, hi=12, vr=6, seed=41)
    T_max = 60
    wmd, T, rho = _conv(vecs, c, q_ids, q_w, 10.0, T_max, tol)
    assert T.min() >= 1 and T.min() < T_max          # the rule does stop some documents
    xs = [np.full((len(q_ids), c.N), 1.0 / len(q_ids))]
    for k in range(1, T_max + 1):
        _, st = _sparse(vecs, c, q_ids, q_w, 10.0, k, return_state=True)
        xs.append(1.0 / st["u"])
    for j in range(c.N):
        ch = [np.max(np.abs(xs[k][:, j] - xs[k - 1][:, j]) / xs[k - 1][:, j]) for k in range(1, T[j] + 1)]
        np.testing.assert_allclose(rho[:T[j], j], ch, rtol=1e-9)
        assert all(v > tol for v in ch[:-1])
        assert ch[-1] <= tol or T[j] == T_max
        assert np.all(np.isnan(rho[T[j]:, j]))
        np.testing.assert_allclose(wmd[j], _sparse(vecs, c, q_ids, q_w, 10.0, int(T[j]), docs=[j])[0],
                                   rtol=1e-12)


def test_one_query_word_stops_after_one_body():
    """v_r = 1: x^(1) = x^(0) sum_w c_wj / r, so x stops changing after one body
    (to the rounding of the float32 weights) and WMD_j = sum_w c_wj m(q, w)."""
    vecs, c, _, _ = _small_problem(seed=43)
    q = 11
    wmd, T, _ = _conv(vecs, c, np.array([q], np.int32), np.array([1.0], np.float32), 10.0, 30, 1e-6)
    assert np.all(T == 1)
    M1 = scipy.spatial.distance.cdist(vecs[[q]].astype(np.float64), vecs.astype(np.float64))[0]
    want = np.array([np.sum(c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]].astype(np.float64)
                            * M1[c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]]]) for j in range(c.N)])
    np.testing.assert_allclose(wmd, want, rtol=1e-12)


def test_iterations_grow_as_tolerance_shrinks_and_cap_holds():
    vecs, c, q_ids, q_w = _small_problem(N=10, seed=47)
    prev = None
    for tol in [1e-1, 1e-2, 1e-3, 1e-5]:
        _, T, _ = _conv(vecs, c, q_ids, q_w, 10.0, 40, tol)
        assert T.max() <= 40
        if prev is not None:
            assert np.all(T >= prev)
        prev = T
    with pytest.raises(ValueError):
        _conv(vecs, c, q_ids, q_w, 10.0, 40, 1.0)


def test_converged_stop_matches_entropic_dual_solution():
    """With a tight tolerance the stopped result is the Sinkhorn fixed point,
    the same <P*, M> that the L-BFGS dual solution of the test above gives."""
    V, d = 12, 10
    vecs = synth.make_vecs(V, d, 4)
    q_ids = np.array([0, 2, 4], np.int32)
    q_w = np.array([0.25, 0.5, 0.25], np.float32)
    c = _one_doc_corpus(V, [5, 7, 9, 11], [0.125, 0.375, 0.25, 0.25])
    lam = 3.0
    got, T, _ = _conv(vecs, c, q_ids, q_w, lam, 5000, 1e-14)
    assert T[0] < 5000
    r = q_w.astype(np.float64)
    cv = c.doc_vals.astype(np.float64)
    M = scipy.spatial.distance.cdist(vecs[q_ids].astype(np.float64), vecs[c.doc_words].astype(np.float64))

    def negdual(z):
        f, g = z[:3], z[3:]
        P = np.exp(lam * (f[:, None] + g[None, :] - M))
        return -(f @ r + g @ cv - P.sum() / lam), -np.concatenate([r - P.sum(1), cv - P.sum(0)])

    res = scipy.optimize.minimize(negdual, np.zeros(7), jac=True, method="L-BFGS-B",
                                  options=dict(ftol=1e-15, gtol=1e-13, maxiter=10000))
    f, g = res.x[:3], res.x[3:]
    P = np.exp(lam * (f[:, None] + g[None, :] - M))
    np.testing.assert_allclose(got, np.sum(P * M), rtol=1e-7)


def test_empty_document_runs_to_the_cap():
    vecs, c, q_ids, q_w = _small_problem(seed=53)
    docs = [(c.doc_words[c.doc_ptr[j]:c.doc_ptr[j + 1]], c.doc_vals[c.doc_ptr[j]:c.doc_ptr[j + 1]]) for j in range(c.N)]
    docs.insert(1, (np.zeros(0, np.int32), np.zeros(0, np.float32)))
    c2 = synth.corpus_from_docs(c.V, docs)
    wmd, T, _ = _conv(vecs, c2, q_ids, q_w, 10.0, 25, 1e-2)
    assert T[1] == 25 and np.isnan(wmd[1])


def test_planted_off_by_one_stop_is_caught():
    """Stopping one body after the rule fires (a classic loop-condition slip)
    is rejected by the relative-change pin."""
    vecs, c, q_ids, q_w = _small_problem(V=80, N=9, lo=3, hi=12, vr=6, seed=41)
    wmd, T, _ = _conv(vecs, c, q_ids, q_w, 10.0, 60, 1e-2)
    late = np.minimum(T + 1, 60)
    bad, _, _ = _conv(vecs, c, q_ids, q_w, 10.0, 60, 0.0, iters=late)
    j = int(np.argmax(T < 60))
    want = _sparse(vecs, c, q_ids, q_w, 10.0, int(T[j]), docs=[j])[0]
    assert abs(bad[j] - want) > 1e-12 * abs(want)


# ---------------------------------------------------------------- k nearest documents
def test_nearest_documents_against_repeated_minimum():
    """Brute force: pick the smallest remaining (NaN last, ties to the lower
    id) k times; -0 and +0 tie."""
    rng = np.random.default_rng(5)
    w = rng.choice([0.5, 1.25, 1.25, 2.0, -0.0, 0.0, np.nan, np.inf, -1.0], 40)
    for k in (1, 5, 17, 40):
        ids, vals = orc.nearest_documents(w, k)
        left = list(range(w.size))
        want = []
        for _ in range(k):
            best = left[0]
            for j in left[1:]:
                a, b = w[j], w[best]
                if np.isnan(b) and not np.isnan(a):
                    best = j
                elif not np.isnan(a) and not np.isnan(b) and a < b:
                    best = j
            want.append(best)
            left.remove(best)
        assert ids.tolist() == want
        assert np.array_equal(vals, w[want], equal_nan=True)


def test_nearest_documents_matches_a_stable_sort():
    """Against numpy's stable argsort (an independent ordering routine): NaN
    sorts last there too, and a stable sort keeps equal values in id order."""
    rng = np.random.default_rng(6)
    w = np.round(rng.random(500) * 20) / 4
    w[rng.choice(500, 30, replace=False)] = np.nan
    w[w == 0] = -0.0
    ids, _ = orc.nearest_documents(w, 200)
    assert ids.tolist() == np.argsort(w + 0.0, kind="stable")[:200].tolist()
