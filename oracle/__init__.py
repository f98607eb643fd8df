"""Plain FP64 CPU oracle for the DMRG operator rotation.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  The
product path (``paper_0909_5662_gb300``) never imports it and shares no code
with it.

Every function restates a definition from Rincon, Garcia and Hallberg,
"Improved parallelization techniques for the density matrix renormalization
group": Sec. 2 step 5 (rotation and decimation R [B a] R^+), the paragraph
after it (blocking Z_[B a] <- Z_[B (+) a], i.e. O (x) I_d), Sec. 3.2 (the two
matrix products Z R^+ then R (Z R^+), the correlation functions <Z_i>,
<Z_i Z_j>, the UMD operator split) and Sec. 3.1 Eq. (hache) (operators
labelled by quantum numbers).

Parity status: every function here is pinned by a test in
``tests/test_oracle_pins.py`` against facts that do not come from the oracle
(closed forms, invariants, brute-force Jordan-Wigner matrix elements, finite
differences).
"""
from .oracle import (  # noqa: F401
    build,
    library_path,
    num_threads,
    rotate_dense,
    rotate_dense_kron,
    rotate_site,
    rotate_site_kron,
    orthonormality_error,
    correlations,
    expectation,
    cross_correlations,
    structure_factor,
    truncation,
    rotate_backward,
    rotate_blocked,
    rotate_blocked_assembled,
    blocked_dense_assembly,
)
