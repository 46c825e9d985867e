"""The projection loop of Sec. 3.1 (Zalesak's disk) on the GPU: the midpoint move with the mesh
velocity (Sec. 3.2 scheme) against the oracle's, the incremental re-binning against the full
binning (bit for bit), and several whole loop steps (M2P -> move -> re-bin -> P2M) against the
oracle running the same steps in FP64."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    return P


def rotation_field(n, omega=2 * np.pi, radius=0.45):
    """Rigid rotation about (0.5, 0.5) within `radius` (the paper rotates the region within 0.9
    of the centre of its (-1, 1)^2 box, period 1), zero outside, at the mesh nodes."""
    g = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(g, g)
    r = np.hypot(X - 0.5, Y - 0.5)
    inside = r < radius
    return np.stack([np.where(inside, -omega * (Y - 0.5), 0.0),
                     np.where(inside, omega * (X - 0.5), 0.0)], -1)


def test_midpoint_move_matches_oracle(P):
    """Random mesh velocity, uniform random particles: FP64 positions after one midpoint step
    within 1e-15 of the oracle's (minimal image); FP32 within 2e-7."""
    n, N = 33, 5000
    pos = G.uniform01(G.SEED_BASE + 510, 2 * N).reshape(N, 2)
    vel = np.random.default_rng(3).standard_normal((n, n, 2))
    vel[-1], vel[:, -1] = vel[0], vel[:, 0]
    ref = O.advect_midpoint(n, pos, vel, 0.01)
    proj = P.Projector(n, N, pos_dtype=torch.float64)
    for dt_, tol in ((torch.float64, 1e-15), (torch.float32, 2e-7)):
        p = torch.tensor(pos, dtype=dt_, device="cuda")
        got = proj.advect(p, torch.tensor(vel, dtype=dt_, device="cuda"), 0.01).double().cpu().numpy()
        d = got - ref
        assert np.abs(d - np.rint(d)).max() <= tol, dt_
        assert (got >= 0).all() and (got < 1).all()


def test_incremental_rebinning_equals_full_binning(P):
    """Jittered lattice moved by random displacements below one bin: the incremental update
    gives the cell list, permutation, sorted positions and fixed point of pfem_build_cells bit
    for bit, for FP64 and FP32 positions, on two consecutive moves."""
    n, M = 65, 128
    pos0 = G.jittered_lattice(M, 0.25, G.SEED_BASE + 511)
    rng = np.random.default_rng(5)
    for dt_ in (torch.float64, torch.float32):
        proj = P.Projector(n, M * M, pos_dtype=dt_)
        ref = P.Projector(n, M * M, pos_dtype=dt_)
        pos = pos0.copy()
        proj.build(torch.tensor(pos, dtype=dt_, device="cuda"))
        bw = 1.0 / proj.nb
        for _ in range(2):
            pos = pos + rng.uniform(-0.9 * bw, 0.9 * bw, pos.shape)
            pos -= np.floor(pos)
            p = torch.tensor(pos, dtype=dt_, device="cuda")
            proj.update(p)
            ref.build(p)
            code, _ = proj.status()
            assert code == 0
            for a, b in ((proj.cells.cell_start, ref.cells.cell_start), (proj.cells.perm, ref.cells.perm),
                         (proj.cells.pos_sorted, ref.cells.pos_sorted),
                         (proj.cells.q_sorted, ref.cells.q_sorted)):
                assert torch.equal(a, b)


def test_incremental_rebinning_flags_a_long_move(P):
    """A particle moved two bins: the update records PFEM_ERR_CAPACITY with the particle's
    index (its outputs are not valid; pfem_build_cells is the remedy), and nothing faults."""
    n, M = 33, 64
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 512)
    proj = P.Projector(n, M * M, pos_dtype=torch.float64)
    proj.build(torch.tensor(pos, device="cuda"))
    moved = pos.copy()
    moved[777, 0] = (moved[777, 0] + 2.5 / proj.nb) % 1.0
    proj.update(torch.tensor(moved, device="cuda"))
    code, detail = proj.status()
    assert code == 4 and detail == 777
    proj.reset_status()
    proj.build(torch.tensor(moved, device="cuda"))
    assert proj.status()[0] == 0


def oracle_loop(n, pos, mesh, vel, dt, steps, m2p_shape, p2m_shape):
    for _ in range(steps):
        vals = O.m2p_quadratic(n, pos, mesh) if m2p_shape == 1 else O.m2p(n, pos, mesh)
        pos = O.advect_midpoint(n, pos, vel, dt)
        mesh = O.p2m(n, pos, vals, shape=p2m_shape, nthreads=8)
    return pos, mesh


@pytest.mark.parametrize("m2p_shape,p2m_shape", [(0, 0), (1, 0), (1, 1)])
def test_zalesak_loop_matches_oracle(P, m2p_shape, p2m_shape):
    """Zalesak's slotted disk on the 65^2 mesh with 64^2 particles, rotation velocity at the
    nodes, dt = 1/160 of a revolution: four whole steps of the library loop (FP64, incremental
    re-binning) against the oracle running the same steps.  Particle positions within 1e-14 and
    the mesh field within 1e-12 of its maximum; the loop with full re-binning gives the same
    result bit for bit."""
    n, M, steps, dt = 65, 64, 4, 1.0 / 160
    g = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(g, g)
    mesh0 = G.zalesak_disk(np.stack([X, Y], -1).reshape(-1, 2)).reshape(n, n, 1)
    pos0 = G.jittered_lattice(M, 0.25, G.SEED_BASE + 90)
    vel = rotation_field(n)
    ref_pos, ref_mesh = oracle_loop(n, pos0, mesh0, vel, dt, steps, m2p_shape, p2m_shape)
    out = []
    for incremental in (True, False):
        proj = P.Projector(n, M * M, C=1, pos_dtype=torch.float64)
        pos = torch.tensor(pos0, device="cuda")
        proj.build(pos)
        pos, mesh = P.projection_loop(proj, pos, torch.tensor(mesh0, device="cuda"),
                                      torch.tensor(vel, device="cuda"), dt, steps,
                                      m2p_shape=m2p_shape, p2m_shape=p2m_shape,
                                      incremental=incremental)
        proj.check()
        out.append((pos, mesh))
        d = pos.cpu().numpy() - ref_pos
        assert np.abs(d - np.rint(d)).max() <= 1e-14
        err = np.abs(mesh.cpu().numpy() - ref_mesh).max() / np.abs(ref_mesh).max()
        assert err <= 1e-12, err
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_host_round_trip_matches_device_steps(P):
    """HostRoundTrip (input copies on their own stream into two alternating buffer sets, P2M
    waiting on the values event before its first kernel that reads the values, results copied
    back on a third stream) returns, step after step, the particle values of build -> P2M -> M2P
    on device-resident inputs, bit for bit; two input sets alternate so that every buffer
    hand-over is exercised."""
    n, M, C = 129, 256, 3
    sets = []
    for k in range(2):
        pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 520 + k).astype(np.float32)
        vals = G.taylor_green(pos.astype(np.float64), k=2 + k).astype(np.float32)
        sets.append((torch.tensor(pos).pin_memory(), torch.tensor(vals).pin_memory()))
    proj = P.Projector(n, M * M, C=C, pos_dtype=torch.float32, ctx=P.Context())
    ref = []
    for pos_h, vals_h in sets:
        pos_d, vals_d = pos_h.cuda(), vals_h.cuda()
        proj.build(pos_d)
        mesh = proj.p2m(vals_d, solve=P.PFEM_SOLVE_F32_REFINED)
        ref.append(proj.m2p(pos_d, mesh).cpu())
    rt = P.HostRoundTrip(proj, C, solve=P.PFEM_SOLVE_F32_REFINED)
    outs = [torch.empty((M * M, C), dtype=torch.float32).pin_memory() for _ in range(6)]
    for k, out_h in enumerate(outs):
        rt.step(*sets[k % 2], out_h)
    rt.inputs_copied()
    rt.wait()
    proj.check()
    for k, out_h in enumerate(outs):
        assert torch.equal(out_h, ref[k % 2]), k
