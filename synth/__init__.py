"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This package holds no arithmetic of the SV-LCOV method itself: it only draws
matrices and update batches (and the starting rank-k factors, which are an
input of every update step) from fixed seeds.
"""
from .generators import (  # noqa: F401
    CSR, csr_from_coo, csr_to_scipy, rng,
    c1_problem, c2_problem, c3_problem, c4_problem, c5_problem, distinct_nonempty_rows,
    chung_lu_edges, init_factors, lookahead_batches, random_csr_batch, random_start,
)
