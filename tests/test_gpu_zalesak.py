"""The paper's Zalesak procedure (Sec. 3.1) through the library loop: every step projects the
slotted-disk indicator mesh -> particles, moves the particles with the midpoint velocity
interpolated from the mesh rotation field (Sec. 3.2 scheme), re-bins them incrementally and
projects particles -> mesh, for one revolution (160 steps).  Linear FE on both sides must
lose more of the disk than mesh QCSF with linear particles, which must lose more than QCSF on
both sides (the ordering of the paper's Fig. zalesak, coarse row, h = H)."""
import json
import os

import numpy as np
import pytest
import torch

from workloads import generators as G

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rotation_field(n, omega=2 * np.pi, radius=0.45):
    """Rigid rotation about (0.5, 0.5) within `radius` (the paper rotates the region within 0.9
    of the centre of its (-1, 1)^2 box, period 1), zero outside, at the mesh nodes."""
    g = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(g, g)
    inside = np.hypot(X - 0.5, Y - 0.5) < radius
    return np.stack([np.where(inside, -omega * (Y - 0.5), 0.0),
                     np.where(inside, omega * (X - 0.5), 0.0)], -1)


def run(P, n, M, mesh_shape, particle_shape, steps):
    g = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(g, g)
    mesh0 = torch.tensor(G.zalesak_disk(np.stack([X, Y], -1).reshape(-1, 2)).reshape(n, n, 1),
                         device="cuda")
    pos = torch.tensor(G.jittered_lattice(M, 0.25, G.SEED_BASE + 90), device="cuda")
    proj = P.Projector(n, M * M, C=1, pos_dtype=torch.float64)
    proj.build(pos)
    _, mesh = P.projection_loop(proj, pos, mesh0.clone(), torch.tensor(rotation_field(n), device="cuda"),
                                1.0 / steps, steps, m2p_shape=mesh_shape, p2m_shape=particle_shape)
    proj.check()
    return (mesh - mesh0).abs().mean().item()


def test_zalesak_rotation_ordering():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    gold = json.load(open(os.path.join(GOLDEN, "zalesak_rotation.json")))
    n, M, steps = 65, 64, 160
    L, Q = P.PFEM_SHAPE_LINEAR, P.PFEM_SHAPE_QUADRATIC
    err = {"fe_fe": run(P, n, M, L, L, steps), "qcsf_fe": run(P, n, M, Q, L, steps),
           "qcsf_qcsf": run(P, n, M, Q, Q, steps)}
    print("Zalesak, mean |alpha - alpha_0| after one revolution:", err)
    order = gold["expected_order_of_error_after_one_revolution"]
    assert err[order[0]] > err[order[1]] > err[order[2]]
