"""Precision study at full size (4097^2 mesh, 8192^2 particles = 67M, Rayleigh-Taylor density):
FP32 and BF16-storage values, each with the FP64 moment solve, the FP32 solve and the FP32
solve with one FP64-residual refinement step; errors against the FP64 oracle on sampled
nodes are printed and bounded."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import generators as G

pytestmark = pytest.mark.gpu


def test_precision_variants_full_size():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    pr = G.config_precision()
    pos = torch.tensor(pr.pos, dtype=torch.float32, device="cuda")
    proj = P.Projector(pr.n, pr.N, C=1, pos_dtype=torch.float32)
    proj.build(pos)
    pos32 = pr.pos.astype(np.float32).astype(np.float64)
    cells = O.build_cells(pr.n, pos32)
    rng = np.random.default_rng(3)
    nodes = rng.choice(pr.n * pr.n, 40, replace=False)
    # nodes near the interface, where the field varies fastest
    J = (0.5 * (pr.n - 1)) + rng.integers(-3, 4, 8)
    I = rng.integers(0, pr.n, 8)
    nodes = np.concatenate([nodes, (J * pr.n + I).astype(np.int64)])
    ref = []
    for node in nodes:
        j, i = divmod(int(node), pr.n)
        idx, w, _, _ = O.node_weights(cells, i, j, 1)
        ref.append(w @ pr.vals[idx, 0])
    ref = np.array(ref)
    scale = np.abs(pr.vals).max()
    errs = {}
    for vt in (torch.float32, torch.bfloat16):
        v = torch.tensor(pr.vals, dtype=torch.float32, device="cuda").to(vt)
        for solve, name in ((P.PFEM_SOLVE_F64, "f64"), (P.PFEM_SOLVE_F32, "f32"),
                            (P.PFEM_SOLVE_F32_REFINED, "f32+ref")):
            m = proj.p2m(v, shape=P.PFEM_SHAPE_QUADRATIC, solve=solve)
            code, _ = proj.status()
            assert code == 0
            got = m.float().cpu().numpy().reshape(-1)[nodes]
            errs[(str(vt), name)] = float(np.abs(got - ref).max() / scale)
    print("precision study, max error / max|rho| vs FP64 oracle:", errs)
    for (vt, _), e in errs.items():
        assert e < (2e-6 if "float32" in vt else 1e-2), errs
