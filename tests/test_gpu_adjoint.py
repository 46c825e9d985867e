"""GPU parity of the adjoint (P2M and M2P backward) against the FP64 oracle's gradients
(complex step for P2M positions, transposed weights for values), central differences of the
GPU forward, and the autograd wrappers."""
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


def relerr(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def small():
    n, M = 17, 32
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 70)
    vals = G.taylor_green(pos)[:, :2].copy()
    g = np.random.default_rng(1).standard_normal((n, n, 2))
    return n, pos, vals, g


def gpu_proj(P, n, pos, C, dtype=torch.float64):
    proj = P.Projector(n, pos.shape[0], C=C, pos_dtype=dtype)
    proj.build(torch.tensor(pos, dtype=dtype, device="cuda"))
    return proj


@pytest.mark.parametrize("shape", [0, 1])
def test_p2m_backward_fp64_matches_oracle(P, small, shape):
    n, pos, vals, g = small
    proj = gpu_proj(P, n, pos, 2)
    gv, gp = proj.backward(torch.tensor(vals, device="cuda"), torch.tensor(g, device="cuda"),
                           shape=shape)
    code, _ = proj.backward_status()
    assert code == 0
    ov, op = O.p2m_backward(n, pos, vals, g, shape=shape)
    ev, ep = relerr(gv.cpu().numpy(), ov), relerr(gp.cpu().numpy(), op)
    print(f"FP64 P2M adjoint vs oracle (shape {shape}): values {ev:.2e}, positions {ep:.2e}")
    assert ev <= 1e-12
    assert ep <= 1e-12


def test_checkpoint_equals_recompute(P, small):
    n, pos, vals, g = small
    proj = gpu_proj(P, n, pos, 2)
    v = torch.tensor(vals, device="cuda")
    gt = torch.tensor(g, device="cuda")
    r_v, r_p = proj.backward(v, gt)
    w = proj.shape_weights(K=32)
    c_v, c_p = proj.backward(v, gt, weights=w)
    assert relerr(c_v.cpu().numpy(), r_v.cpu().numpy()) <= 1e-13
    assert relerr(c_p.cpu().numpy(), r_p.cpu().numpy()) <= 1e-13
    c_v2, c_p2 = proj.backward(v, gt, weights=w, want_pos=False)
    assert c_p2 is None and torch.equal(c_v2, c_v)


def test_value_gradient_dot_product(P, small):
    n, pos, vals, g = small
    proj = gpu_proj(P, n, pos, 2)
    a = torch.tensor(np.random.default_rng(3).standard_normal(vals.shape), device="cuda")
    gt = torch.tensor(g, device="cuda")
    gv, _ = proj.backward(a, gt, want_pos=False)
    lhs = (proj.p2m(a) * gt).sum().item()
    assert abs(lhs - (a * gv).sum().item()) <= 1e-12 * abs(lhs)


def test_position_gradient_vs_gpu_central_differences(P, small):
    """Central differences (step 1e-6, FP64) of the GPU forward; samples whose stencils
    change between the two evaluations are skipped and counted."""
    n, pos, vals, g = small
    proj = gpu_proj(P, n, pos, 2)
    v = torch.tensor(vals, device="cuda")
    gt = torch.tensor(g, device="cuda")
    _, gp = proj.backward(v, gt)
    gp = gp.cpu().numpy()
    rng = np.random.default_rng(9)
    ok = 0
    for m in rng.choice(pos.shape[0], 24, replace=False):
        for dim in (0, 1):
            vals_pm, sets = [], []
            for sgn in (1, -1):
                p2 = pos.copy()
                p2[m, dim] += sgn * 1e-6
                pr = gpu_proj(P, n, p2, 2)
                vals_pm.append((pr.p2m(v) * gt).sum().item())
                wi, _ = pr.shape_weights(K=32)
                perm = pr.cells.perm.cpu().numpy()
                wi = wi.cpu().numpy()
                sets.append([tuple(sorted(perm[r[r >= 0]])) for r in wi])
            if sets[0] != sets[1]:
                continue
            fd = (vals_pm[0] - vals_pm[1]) / 2e-6
            assert abs(fd - gp[m, dim]) <= 1e-6 * max(1.0, abs(fd)), (m, dim, fd, gp[m, dim])
            ok += 1
    assert ok >= 30


def test_m2p_backward_matches_oracle(P, small):
    n, pos, _, _ = small
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n, n, 3))
    gv = rng.standard_normal((pos.shape[0], 3))
    proj = gpu_proj(P, n, pos, 3)
    gm, gp = proj.m2p_backward(torch.tensor(pos, device="cuda"), torch.tensor(f, device="cuda"),
                               torch.tensor(gv, device="cuda"))
    om, op = O.m2p_backward(n, pos, f, gv)
    assert relerr(gm.cpu().numpy(), om) <= 1e-12
    assert relerr(gp.cpu().numpy(), op) <= 1e-12


def test_autograd_round_trip(P, small):
    """loss(P2M -> M2P) differentiated by torch.autograd through both Functions equals the
    composition of the direct adjoint calls."""
    n, pos, vals, g = small
    pos_t = torch.tensor(pos, device="cuda", requires_grad=True)
    v_t = torch.tensor(vals, device="cuda", requires_grad=True)
    mesh = P.autograd.p2m(v_t, pos_t, n)
    back = P.autograd.m2p(mesh, pos_t, n)
    target = torch.tensor(np.random.default_rng(8).standard_normal(back.shape), device="cuda")
    loss = 0.5 * ((back - target) ** 2).sum()
    gv, gp = torch.autograd.grad(loss, (v_t, pos_t))
    # direct composition
    proj = gpu_proj(P, n, pos, 2)
    m2 = proj.p2m(torch.tensor(vals, device="cuda"))
    b2 = proj.m2p(torch.tensor(pos, device="cuda"), m2)
    gb = b2 - target
    gm, gp_m2p = proj.m2p_backward(torch.tensor(pos, device="cuda"), m2, gb)
    gv2, gp_p2m = proj.backward(torch.tensor(vals, device="cuda"), gm)
    assert relerr(gv.cpu().numpy(), gv2.cpu().numpy()) <= 1e-14
    assert relerr(gp.cpu().numpy(), (gp_m2p + gp_p2m).cpu().numpy()) <= 1e-14


def test_fp32_backward_error_against_fp64_oracle(P, small):
    n, pos, vals, g = small
    pos32 = pos.astype(np.float32).astype(np.float64)
    ov, op = O.p2m_backward(n, pos32, vals, g, shape=1)
    proj = gpu_proj(P, n, pos32, 2, torch.float32)
    errs = {}
    for solve, name in ((P.PFEM_SOLVE_F32, "f32"), (P.PFEM_SOLVE_F64, "f64")):
        gv, gp = proj.backward(torch.tensor(vals, dtype=torch.float32, device="cuda"),
                               torch.tensor(g, dtype=torch.float32, device="cuda"), solve=solve)
        errs[name] = (relerr(gv.cpu().numpy(), ov), relerr(gp.cpu().numpy(), op))
    print("FP32 backward error vs FP64 oracle (vals, pos):", errs)
    for ev, ep in errs.values():
        assert ev < 1e-5 and ep < 1e-2


def test_gradient_workload_full_size_band(P):
    """Gradient workload at full size (1025^2 mesh, 2048^2 particles, FP32 launch as timed):
    the upstream gradient is restricted to a band of 6 node rows, so the oracle (complex step)
    only has to visit those nodes; every particle's gradient is compared."""
    pr = G.config_grad()
    n = pr.n
    rows = slice(500, 506)
    rng = np.random.default_rng(12)
    g = np.zeros((n, n, 1))
    g[rows] = rng.standard_normal((6, n, 1))
    pos32 = pr.pos.astype(np.float32).astype(np.float64)
    ov, op = O.p2m_backward(n, pos32, pr.vals, g, shape=1, node_range=(500 * n, 506 * n))
    res = {}
    for dt in (torch.float64, torch.float32):
        proj = gpu_proj(P, n, pos32, 1, dt)
        gv, gp = proj.backward(torch.tensor(pr.vals, dtype=dt, device="cuda"),
                               torch.tensor(g, dtype=dt, device="cuda"))
        code, _ = proj.backward_status()
        assert code == 0
        res[str(dt)] = (relerr(gv.cpu().numpy(), ov), relerr(gp.cpu().numpy(), op))
    print("full-size band gradient error (vals, pos):", res)
    assert res["torch.float64"][0] <= 1e-12 and res["torch.float64"][1] <= 1e-12
    assert res["torch.float32"][0] < 1e-5 and res["torch.float32"][1] < 1e-2


def test_uniform_random_gradient_takes_the_fix_pass(P):
    """Uniform random particles (512^2 on the 257^2 mesh): the node rows 40..63 include node
    (68, 52), whose edge stencil of five particles makes its system inconsistent (least
    squares, rank 5), and edge systems too ill-conditioned for the fast FP32 solve.  Those nodes
    go to the adjoint's fix pass (FP64, derivative of the SVD pseudo-inverse with the edge frame
    differentiated); no device error.  The upstream gradient is non-zero on those rows only,
    and every particle's value and position gradient is compared with the oracle's (complex
    step through its own least-squares route).  FP64 values within 1e-12.  FP64 positions within
    1e-10, a bound set by conditioning: for full-rank stencils both sides differentiate the
    normal equations of the 6 x 6 moment matrix (the GPU's Cholesky keeps systems whose pivots
    stay above 1e-6 of the trace, so kappa(M) <= ~1e6; the oracle's complex-symmetric Cholesky
    has the same sensitivity), so a node's position derivatives carry errors up to
    kappa(M) eps64 ~ 1e-10 (measured 3.2e-11 here; the jittered lattices, kappa <= ~1e3, stay
    within 1e-12).  FP32 values within 1e-5 and positions within 1e-2 of the largest entry."""
    n, M = 257, 512
    N = M * M
    pos = G.uniform01(G.SEED_BASE + 62, 2 * N).reshape(N, 2)
    vals = G.taylor_green(pos)[:, :2].copy()
    g = np.zeros((n, n, 2))
    g[40:64] = np.random.default_rng(31).standard_normal((24, n, 2))
    res = {}
    for dt in (torch.float64, torch.float32):
        p = pos if dt == torch.float64 else pos.astype(np.float32).astype(np.float64)
        ov, op = O.p2m_backward(n, p, vals, g, shape=1, node_range=(40 * n, 64 * n))
        proj = gpu_proj(P, n, p, 2, dt)
        solve = P.PFEM_SOLVE_F64 if dt == torch.float64 else P.PFEM_SOLVE_F32
        gv, gp = proj.backward(torch.tensor(vals, dtype=dt, device="cuda"),
                               torch.tensor(g, dtype=dt, device="cuda"), solve=solve)
        code, detail = proj.backward_status()
        assert code == 0, (dt, detail)
        res[str(dt)] = (relerr(gv.cpu().numpy(), ov), relerr(gp.cpu().numpy(), op))
    print("uniform random gradient error (vals, pos):", res)
    assert res["torch.float64"][0] <= 1e-12 and res["torch.float64"][1] <= 1e-10
    assert res["torch.float32"][0] < 1e-5 and res["torch.float32"][1] < 1e-2
