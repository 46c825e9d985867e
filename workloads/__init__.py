"""Seeded synthetic inputs for the particle <-> fixed-mesh projection round trip.

This module holds no arithmetic of the projection method itself: it only draws
particle positions on a jittered lattice of the unit periodic square and
evaluates the analytic fields the paper's experiments use (Taylor-Green vortex
sheet, Zalesak slotted disk, Rayleigh-Taylor density step).  Both the CUDA path
and the CPU oracle take their inputs from here, and nothing else is shared.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written from its published
definition and vectorised with numpy's wrapping uint64 arithmetic.
"""
from .generators import (  # noqa: F401
    SEED_BASE,
    splitmix64,
    uniform01,
    jittered_lattice,
    taylor_green,
    zalesak_disk,
    rayleigh_taylor,
    Problem,
    config_tiny,
    config_large,
    config_precision,
    config_batched,
    config_grad,
    scaled_config,
    six_per_node,
    particles_at_nodes,
)
