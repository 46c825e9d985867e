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


def test_full_size_batched_workload_sampled(P):
    """The batched workload at full size (256 problems, 2.0e8 particles, FP32, graph replay in
    the tuned configuration as benchmarked): three sampled problems equal their single-problem
    runs bit for bit, and one of them matches the FP64 oracle at sampled nodes within FP32
    error."""
    probs = G.config_batched()
    b, pos, vals = make_batch(P, probs, torch.float32)
    from paper_1610_05266_gb300 import tuner
    tuner.tune_batch(b, pos, vals, P.PFEM_SHAPE_QUADRATIC, quick=True)
    b.capture(pos, vals)
    back = b.replay()
    torch.cuda.synchronize()
    code, _ = b.status()
    assert code == 0
    rng = np.random.default_rng(4)
    picks = sorted(rng.choice(len(probs), 3, replace=False))
    for p in picks:
        mesh1, back1 = single(P, probs[p], torch.float32, 1)
        assert torch.equal(b.mesh_view(p), mesh1), p
        assert torch.equal(back[b.offsets[p]: b.offsets[p + 1]], back1), p
    pr = probs[picks[0]]
    pos32 = pr.pos.astype(np.float32).astype(np.float64)
    cells = O.build_cells(pr.n, pos32)
    m = b.mesh_view(picks[0]).cpu().numpy()
    worst = 0.0
    for node in rng.choice(pr.n * pr.n, 32, replace=False):
        J, I = divmod(int(node), pr.n)
        idx, w, _, _ = O.node_weights(cells, I, J, 1)
        worst = max(worst, np.abs(m[J, I] - w @ pr.vals[idx]).max())
    assert worst / np.abs(pr.vals).max() < 1e-5
