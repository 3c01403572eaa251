"""FP64 CPU oracle for the sparse Sinkhorn-Knopp WMD.

Test infrastructure: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  See ``oracle/sinkhorn_wmd.py``.
"""
from .sinkhorn_wmd import (  # noqa: F401
    select_nonzero,
    cdist,
    sinkhorn_wmd_dense,
    sinkhorn_wmd_sparse,
    sinkhorn_wmd_sparse_until_converged,
    nearest_documents,
    emd_uniform_bruteforce,
)
