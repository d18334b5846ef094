"""FP64 CPU oracle of the Cascade-of-Gaussians step (arXiv 1705.09339).

Test infrastructure only: the test suite, the smoke check and the
benchmark's CPU-baseline leg are its only users.  The product package never
imports it.  See ``cog_oracle.h`` for what each routine follows in the paper.
"""
from .oracle import (  # noqa: F401
    ORC_CONF, ORC_FD, ORC_ILLUM, ORC_MODE1, ORC_PERCHAN, ORC_RGA, ORC_SAMPLE, NEAR_BITS, Oracle, OracleState,
    build_oracle, default_params, group_assign, group_centroids, group_cluster, group_cores, group_init, kde_weights,
    oracle_threads, set_threads,
)
