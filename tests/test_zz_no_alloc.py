"""pfem_build_cells_noalloc: the binning for callers that cannot allocate device memory.

It must give exactly what pfem_build_cells gives (integer outputs, so bit for bit), on
consecutive calls that reuse the library's one scratch array.  This file is collected last
so that a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from workloads import generators as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    return P


def _reference(P, pos, nb):
    N = pos.shape[0]
    proj = P.Projector(33, N, nb=nb, pos_dtype=pos.dtype, device=pos.device)
    c = proj.build(pos)
    return [t.clone() for t in (c.cell_start, c.perm, c.pos_sorted, c.q_sorted)]


def _noalloc(P, pos, nb):
    N = pos.shape[0]
    dev = pos.device
    out = [torch.full((nb * nb + 1,), -7, dtype=torch.int32, device=dev),
           torch.full((N,), -7, dtype=torch.int32, device=dev),
           torch.full((N, 2), -7.0, dtype=pos.dtype, device=dev),
           torch.full((N, 2), -7, dtype=torch.int32, device=dev)]
    P.pfem_build_cells_noalloc(nb, N, pos, *out)
    return out


def test_noalloc_matches_workspace_entry_point_on_consecutive_calls(P):
    dev = torch.device("cuda")
    cases = [(G.jittered_lattice(200, 0.25, G.SEED_BASE + 77), 100, torch.float32),
             (G.jittered_lattice(64, 0.3, G.SEED_BASE + 78), 32, torch.float64),
             (G.jittered_lattice(2048, 0.25, G.SEED_BASE + 2), 1024, torch.float32)]
    for pos_np, nb, dt in cases:
        pos = torch.tensor(pos_np, dtype=dt, device=dev)
        ref = _reference(P, pos, nb)
        for _ in range(2):                       # two calls in a row on the shared scratch
            got = _noalloc(P, pos, nb)
            torch.cuda.synchronize()
            for r, g in zip(ref, got):
                assert torch.equal(r, g)


def test_noalloc_rejects_sizes_beyond_its_scratch(P):
    dev = torch.device("cuda")
    pos = torch.zeros((4, 2), dtype=torch.float32, device=dev)
    buf = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(P.PfemError) as e:
        P.pfem_build_cells_noalloc(1025, 4, pos, buf, buf, pos, buf)   # 1025^2 bins > 2^20
    assert e.value.code == 4
    with pytest.raises(P.PfemError) as e:
        P.pfem_build_cells_noalloc(64, (1 << 22) + 1, pos, buf, buf, pos, buf)
    assert e.value.code == 4
