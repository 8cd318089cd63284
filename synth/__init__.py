"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the bench.

This package holds no arithmetic of the layout method itself: it only builds
graphs (symmetric CSR, sorted rows, no self-loops) and initial positions from
numpy's PCG64 generator, so that both sides of a parity check see identical
inputs.
"""
from .graphs import (  # noqa: F401
    Graph,
    edges_to_csr,
    sbm_graph,
    lfr_graph,
    rmat_graph,
    rmat_graph_native,
    batch_sbm_graphs,
    planted_partition_graph,
    serving_graph_pool,
    initial_positions,
    tiny_graph,
    bfs_relabel,
    source_digest,
)
