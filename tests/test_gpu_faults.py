"""Bounded loops, capacities and sparse regions on the GPU: each cap of a context makes its loop
run out and the call report a status through the device status word (no trap, no hang); a void
in the particles, which the first search radius cannot bridge, is recomputed by the wider
retry and fix passes and matches the oracle; with the widest radius capped below the void, the
same input reports PFEM_ERR_CAPACITY."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TIMEOUT, CAPACITY = 6, 4


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    return P


def relerr(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def run(P, pr, ctx=None, shape=1, dtype=torch.float64, solve=None):
    proj = P.Projector(pr.n, pr.N, C=pr.C, pos_dtype=dtype, ctx=ctx)
    proj.build(torch.tensor(pr.pos, dtype=dtype, device="cuda"))
    mesh = proj.p2m(torch.tensor(pr.vals, dtype=dtype, device="cuda"), shape=shape, solve=solve)
    code, detail = proj.status()
    return mesh.cpu().numpy(), code, detail, proj


def void_problem(R=0.08):
    """128^2 jittered lattice on a 65^2 mesh with every particle within R (10 spacings) of the
    centre removed: the void is five bins wide, beyond the first search radius (4 bins)."""
    M, n = 128, 65
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 300)
    d = pos - 0.5
    d -= np.rint(d)
    pos = np.ascontiguousarray(pos[(d ** 2).sum(1) >= R * R])
    return G.Problem("void", n, M, 0.25, 0, pos, G.taylor_green(pos))


@pytest.mark.parametrize("shape", [0, 1])
def test_walk_cap_reports_timeout(P, shape):
    """walk_max_steps = -1 (no step of the visibility walk): the nodes whose nearest particle's
    fan does not contain them (about 5 % on the jittered lattice) record PFEM_ERR_TIMEOUT;
    the default context records nothing."""
    pr = G.config_tiny()
    _, code, detail, _ = run(P, pr, shape=shape)
    assert code == 0
    ctx = P.Context(walk_max_steps=-1)
    _, code, detail, proj = run(P, pr, ctx, shape=shape)
    assert code == TIMEOUT and 0 <= detail < pr.n * pr.n
    assert "iteration cap" in ctx.last_error()


@pytest.mark.parametrize("shape", [0, 1])
def test_star_capacity_reports_capacity(P, shape):
    """star_capacity = 3: every star has more than three Delaunay neighbours, so the star table
    (quadratic) and the per-node search (linear) record PFEM_ERR_CAPACITY."""
    pr = G.config_tiny()
    ctx = P.Context(star_capacity=3)
    _, code, _, _ = run(P, pr, ctx, shape=shape)
    assert code == CAPACITY
    assert "capacity" in ctx.last_error()


def test_node_capacity_sends_every_node_to_the_fix_pass(P):
    """node_capacity = 3: no node's particle set fits the fast pass, so every node is queued and
    recomputed by the fix pass (FP64, SVD solve of each edge); the mesh still matches the
    oracle within 1e-12 and no error is recorded."""
    pr = G.config_tiny()
    mesh, code, _, _ = run(P, pr, P.Context(node_capacity=3))
    assert code == 0
    assert relerr(mesh, O.p2m(pr.n, pr.pos, pr.vals, shape=1, nthreads=8)) <= TOL64


@pytest.mark.parametrize("shape", [0, 1])
def test_void_is_bridged_by_the_wider_passes(P, shape):
    """A void ten particle spacings in radius: nodes inside it find no particle within the first
    search radius, and the stars around it have circumcircles wider than the candidate cutoff.
    The retry kernel (stars) and the fix pass (nodes) search up to a quarter of the torus, in
    the same launch sequence with no host synchronisation; the FP64 mesh matches the oracle
    within 1e-12 and no error is recorded."""
    pr = void_problem()
    mesh, code, detail, _ = run(P, pr, shape=shape)
    assert code == 0, detail
    assert relerr(mesh, O.p2m(pr.n, pr.pos, pr.vals, shape=shape, nthreads=8)) <= TOL64


def test_void_fp32_quadratic(P):
    """The void with FP32 positions and values and the refined FP32 solve: every node within
    2e-6 of the FP64 oracle run on the same FP32 positions."""
    pr = void_problem()
    pos32 = pr.pos.astype(np.float32).astype(np.float64)
    pr32 = G.Problem("void32", pr.n, pr.M, pr.a, 0, pos32, pr.vals)
    mesh, code, _, _ = run(P, pr32, dtype=torch.float32, solve=P.PFEM_SOLVE_F32_REFINED)
    assert code == 0
    ref = O.p2m(pr.n, pos32, pr.vals, shape=1, nthreads=8)
    assert relerr(mesh.astype(np.float64), ref) <= 2e-6


def test_void_with_capped_radius_reports_capacity(P):
    """The same void with search_radius_max = 4 bins (the first radius): the wider passes cannot
    reach across it, so the call records PFEM_ERR_CAPACITY instead of a wrong value."""
    ctx = P.Context(search_radius_max=4)
    _, code, _, _ = run(P, void_problem(), ctx)
    assert code == CAPACITY


def test_device_status_text(P):
    """pfem_get_device_status describes a device error in the context's last-error text."""
    ctx = P.Context(walk_max_steps=-1)
    _, _, _, proj = run(P, G.config_tiny(), ctx, shape=0)
    code, _ = proj.status()
    assert code == TIMEOUT
    assert ctx.last_error().startswith("device status iteration cap reached")
