"""Seeded synthetic inputs for the DMRG operator rotation.

This package only draws random numbers and lays them out: it holds none of
the rotation's arithmetic, so both the CUDA library's tests/benchmark and the
CPU oracle can consume the same bytes.  The paper (Sec. 2.1, Sec. 3.2) runs
DMRG on the quarter-filled 1D Hubbard chain; no dataset exists, so these
generators produce Hubbard-shaped stand-ins: site dimension d = 4 with local
states (0, up, down, up-down), kept-state counts m taken from the paper's
runs (m = 400, m = 1000), truncation matrices with orthonormal columns, and
operator batches sized like the L = l(l+3)/2 stored Z_i, Z_i Z_j operators of
Sec. 3.2.
"""
from .synthetic import (  # noqa: F401
    SEED_BASE,
    DenseWorkload,
    BlockedWorkload,
    orthonormal_columns,
    dense_workload,
    dense_config,
    blocked_config,
    blocked_layout_sizes,
    gaussian_sector_split,
    HUBBARD_SITE_SHIFTS,
    backward_upstream,
    chained_inputs,
    schmidt_state,
    HUBBARD_SITE_OPS,
    SiteWorkload,
    site_workload,
    MeasureWorkload,
    measure_workload,
)
