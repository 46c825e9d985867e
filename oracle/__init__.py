"""Plain FP64 CPU oracle for the particle <-> fixed-mesh projection round trip.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark use it; the CUDA library never does, and the two share no code.
"""
from .oracle import (  # noqa: F401
    build,
    lib,
    build_cells,
    node_weights,
    node_edges,
    node_weight_derivs,
    star,
    p2m,
    m2p,
    m2p_quadratic,
    mesh_edge,
    p2m_backward,
    m2p_backward,
    advect_midpoint,
    fixed_point,
    OracleError,
    KSTEN,
)
