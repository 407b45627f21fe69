"""Seeded synthetic inputs shared by the CUDA path, its tests, the benchmark and the oracle.

This package builds generator sets (permutations in one-line notation) and the seeded job
lists of the batched and serving workloads.  It holds none of the growth method's arithmetic:
no packing, no permutation action, no deduplication.  Both the oracle and the library consume
its output as plain lists of integers.
"""

from .families import (  # noqa: F401
    FAMILIES,
    all_transpositions,
    binary_start,
    consecutive_3cycles_inv,
    consecutive_4cycles,
    coxeter,
    cycle,
    cycles_01i_inv,
    cyclic_coxeter,
    from_cycles,
    identity,
    inverse,
    inverse_closure,
    is_inverse_closed,
    koltsov3,
    lrx,
    lx,
    pancake,
    prefix_cycles,
    random_perms,
    reversals,
    star,
    three_cycles,
    transposons,
)
from .configs import (  # noqa: F401
    BATCH_SEED,
    SERVE_SEED,
    GrowthJob,
    batch_groups,
    config_s8_coxeter,
    config_s11_lrx,
    config_s14_pancake,
    serve_stream,
)
