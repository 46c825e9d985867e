"""Batched persistent launches (many uneven problems at once), CUDA-graph replay and the
autotuner: the batched outputs must equal the single-problem path bit for bit (same
topology and arithmetic), and single problems must match the FP64 oracle."""
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


def make_batch(P, probs, dtype):
    sizes = [(pr.n, pr.N) for pr in probs]
    b = P.Batch(sizes, C=probs[0].C, dtype=dtype)
    pos = torch.tensor(np.concatenate([pr.pos for pr in probs]), dtype=dtype, device="cuda")
    vals = torch.tensor(np.concatenate([pr.vals for pr in probs]), dtype=dtype, device="cuda")
    return b, pos, vals


def single(P, pr, dtype, shape):
    proj = P.Projector(pr.n, pr.N, C=pr.C, pos_dtype=dtype)
    pos = torch.tensor(pr.pos, dtype=dtype, device="cuda")
    proj.build(pos)
    mesh = proj.p2m(torch.tensor(pr.vals, dtype=dtype, device="cuda"), shape=shape)
    back = proj.m2p(pos, mesh)
    proj.check()
    return mesh, back


@pytest.mark.parametrize("dtype,shape", [(torch.float32, 1), (torch.float64, 1), (torch.float32, 0)])
def test_batch_equals_single_problems(P, dtype, shape):
    probs = G.config_batched(count=7, size_scale=0.12)
    b, pos, vals = make_batch(P, probs, dtype)
    for tile_rows in (4, 8, 16):
        b.build(pos)
        b.p2m(vals, shape=shape, tile_rows=tile_rows, blocks=152 * 2)
        back = b.m2p(pos)
        code, _ = b.status()
        assert code == 0
        for p, pr in enumerate(probs):
            mesh1, back1 = single(P, pr, dtype, shape)
            assert torch.equal(b.mesh_view(p), mesh1), (p, tile_rows)
            assert torch.equal(back[b.offsets[p]: b.offsets[p + 1]], back1), p


def test_batch_problem_matches_oracle(P):
    probs = G.config_batched(count=5, size_scale=0.1)
    b, pos, vals = make_batch(P, probs, torch.float64)
    b.round_trip(pos, vals)
    for p in (0, 3):
        pr = probs[p]
        ref = O.p2m(pr.n, pr.pos, pr.vals, shape=1, nthreads=8)
        m = b.mesh_view(p).cpu().numpy()
        assert np.abs(m - ref).max() / np.abs(ref).max() <= 1e-12


def test_graph_replay_and_autotuner(P):
    from paper_1610_05266_gb300 import tuner
    probs = G.config_batched(count=9, size_scale=0.15)
    b, pos, vals = make_batch(P, probs, torch.float32)
    eager = b.round_trip(pos, vals).clone()
    cfg = tuner.tune_batch(b, pos, vals, P.PFEM_SHAPE_QUADRATIC, quick=True)
    assert cfg["tile_rows"] in (4, 8, 16) and cfg["p2m_blocks"] > 0
    b.capture(pos, vals)
    for _ in range(2):
        out = b.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)
    code, _ = b.status()
    assert code == 0


def test_full_size_batched_workload(P):
    """The batched workload at full size (256 problems, 2.0e8 particles, FP32 values, FP32
    Cholesky with one FP64-residual refinement step, graph replay in the tuned configuration as
    benchmarked): three sampled problems equal their single-problem runs bit for bit, and every
    node of those problems matches the FP64 oracle (same FP32 positions) within 1e-6 of
    max|field| per channel."""
    import os
    probs = G.config_batched()
    b, pos, vals = make_batch(P, probs, torch.float32)
    from paper_1610_05266_gb300 import tuner
    sv = P.PFEM_SOLVE_F32_REFINED
    tuner.tune_batch(b, pos, vals, P.PFEM_SHAPE_QUADRATIC, sv, quick=True)
    b.capture(pos, vals, solve=sv)
    back = b.replay()
    torch.cuda.synchronize()
    code, _ = b.status()
    assert code == 0
    rng = np.random.default_rng(4)
    picks = sorted(rng.choice(len(probs), 3, replace=False))
    for p in picks:
        pr = probs[p]
        proj = P.Projector(pr.n, pr.N, C=pr.C, pos_dtype=torch.float32)
        pp = torch.tensor(pr.pos, dtype=torch.float32, device="cuda")
        proj.build(pp)
        mesh1 = proj.p2m(torch.tensor(pr.vals, dtype=torch.float32, device="cuda"), solve=sv)
        back1 = proj.m2p(pp, mesh1)
        proj.check()
        assert torch.equal(b.mesh_view(p), mesh1), p
        assert torch.equal(back[b.offsets[p]: b.offsets[p + 1]], back1), p
        pos32 = pr.pos.astype(np.float32).astype(np.float64)
        ref = O.p2m(pr.n, pos32, pr.vals, shape=1, nthreads=os.cpu_count() or 8)
        m = b.mesh_view(p).cpu().numpy().astype(np.float64)
        err = (np.abs(m - ref).reshape(-1, 3).max(0) / np.abs(ref).reshape(-1, 3).max(0)).max()
        print(f"batch problem {p} (n={pr.n}, N={pr.N}): {err:.2e}")
        assert err < 1e-6, (p, err)


def _uniform(n, N, seed):
    pos = G.uniform01(G.SEED_BASE + seed, 2 * N).reshape(N, 2)
    return G.Problem(f"uniform_{n}_{N}", n, int(np.sqrt(N)), 0.0, 0, pos, G.taylor_green(pos))


def test_uniform_random_batch_takes_the_fix_pass(P):
    """A batch of uniform random (Poisson) particle sets, whose nodes include ill-conditioned
    and rank-deficient edge systems, systems of more than 24 particles and stars wider than the
    candidate cutoff: the batched star table, geometry, solve and fix pass (FP64 SVD solve with
    the problem's own bins) run with no device error.  Problem 0 is 2048^2 particles on the
    1025^2 mesh, where node (245, 118) has a rank-5 edge system; it is checked at that node and
    48 random nodes, the three smaller problems at every node.  FP64: 1e-12 of max|field|;
    FP32 values with the refined solve (same FP32 positions for the oracle): 1e-5."""
    import os
    probs = [_uniform(1025, 2048 * 2048, 62), _uniform(65, 3000, 63), _uniform(97, 40000, 64),
             _uniform(33, 900, 65)]
    rng = np.random.default_rng(7)
    big_nodes = [(245, 118)] + [tuple(int(t) for t in rng.integers(0, 1024, 2)) for _ in range(48)]
    for dtype, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        b, pos, vals = make_batch(P, probs, dtype)
        sv = P.PFEM_SOLVE_F64 if dtype == torch.float64 else P.PFEM_SOLVE_F32_REFINED
        b.round_trip(pos, vals, solve=sv)
        code, detail = b.status()
        assert code == 0, (dtype, detail)
        for p, pr in enumerate(probs):
            ppos = pr.pos if dtype == torch.float64 else pr.pos.astype(np.float32).astype(np.float64)
            m = b.mesh_view(p).cpu().numpy().astype(np.float64)
            vmax = np.abs(pr.vals).max()
            if p == 0:
                cells = O.build_cells(pr.n, ppos)
                for k, (I, J) in enumerate(big_nodes):
                    idx, w, _, rank = O.node_weights(cells, I, J, 1)
                    if k == 0:
                        assert rank == 5
                    assert np.abs(m[J, I] - w @ pr.vals[idx]).max() <= tol * vmax, (dtype, I, J)
            else:
                ref = O.p2m(pr.n, ppos, pr.vals, shape=1, nthreads=os.cpu_count() or 8)
                assert np.abs(m - ref).max() <= tol * vmax, (dtype, p)
