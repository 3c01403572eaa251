"""Host-side logic of bench.py (no GPU): the document sample taken on large
corpora, the all-cores oracle baseline (spawned workers that finish instead of
hanging), and the paper's per-iteration byte count B_iter."""
import numpy as np

import bench
from paper_2005_06727_gb300 import synth


class _Corpus:
    def __init__(self, lengths):
        self.N = len(lengths)
        self.doc_ptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        self.nnz = int(self.doc_ptr[-1])


def test_small_corpora_use_every_document():
    assert bench.oracle_docs(_Corpus(np.full(bench.SAMPLE_ABOVE, 5))) is None


def test_large_corpora_sample_includes_longest_and_shortest():
    rng = np.random.default_rng(1)
    lengths = rng.integers(20, 201, 50_000)
    c = _Corpus(lengths)
    docs = bench.oracle_docs(c)
    assert docs is not None and np.all(np.diff(docs) > 0)
    assert 2000 <= docs.size <= 2040
    assert set(np.argsort(lengths)[-20:]) <= set(docs.tolist())
    assert set(np.argsort(lengths)[:20]) <= set(docs.tolist())
    assert np.array_equal(docs, bench.oracle_docs(c))      # seeded


def test_all_cores_oracle_finishes_and_reports_its_cores():
    w = synth.TINY
    _, c, _ = synth.make_workload(w, 1)
    rec = bench.cpu_baseline_all_cores(w, c, timeout_s=120.0)
    assert rec["kind"] == "oracle" and rec["unit"] == bench.UNIT
    assert rec["value"] > 0 and 1 <= rec["cores"] <= c.N


def test_effective_hbm_is_the_per_iteration_byte_count():
    """B_iter = (T+1) [8 nnz + 4 (N+1) + 8 v_r N] + 8 v_r V + 8 N: the paper's
    per-iteration formulation streams c (ids and values) and the dense u/x
    state in every SDDMM_SpMM pass and reads K and M once."""
    w = synth.PAPER
    c = _Corpus(np.full(w.N, 85))
    v_r, T = 30, w.max_iter
    rec = bench.effective_hbm(w, c, v_r, loop_ms=1.0, step_ms=2.0, peak_gbs=1000.0)
    per_pass = 8 * c.nnz + 4 * (c.N + 1) + 8 * v_r * c.N
    want = (T + 1) * per_pass + 8 * v_r * w.V + 8 * c.N
    assert rec["b_iter_bytes"] == want
    assert abs(rec["loop_gbs"] - want / 1e-3 / 1e9) < 1e-9
    assert abs(rec["step_frac"] - want / 2e-3 / 1e9 / 1000.0) < 1e-12
