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
    """Full size (4097^2 mesh, 8192^2 = 67M particles, RT density): every node of the 16 node
    rows that cross the interface y = 0.5 + 0.05 cos(2 pi x), where the density varies
    fastest (65,552 nodes), against the FP64 oracle run on the same FP32 positions, for FP32 and
    BF16-storage values with each moment solve.  Bounds: FP32 values 1e-6, BF16 values 1e-2
    (measured 3.3e-7 and 4.4e-3: the storage rounding of the values)."""
    import os
    import __graft_entry__
    __graft_entry__.build()
    import paper_1610_05266_gb300 as P
    pr = G.config_precision()
    pos = torch.tensor(pr.pos, dtype=torch.float32, device="cuda")
    proj = P.Projector(pr.n, pr.N, C=1, pos_dtype=torch.float32)
    proj.build(pos)
    J0, J1 = 2040, 2056
    pos32 = pr.pos.astype(np.float32).astype(np.float64)
    ref = O.p2m(pr.n, pos32, pr.vals, shape=1, nthreads=os.cpu_count() or 8,
                node_range=(J0 * pr.n, J1 * pr.n))[J0:J1, :, 0]
    scale = np.abs(ref).max()
    errs = {}
    for vt in (torch.float32, torch.bfloat16):
        v = torch.tensor(pr.vals, dtype=torch.float32, device="cuda").to(vt)
        for solve, name in ((P.PFEM_SOLVE_F64, "f64"), (P.PFEM_SOLVE_F32, "f32"),
                            (P.PFEM_SOLVE_F32_REFINED, "f32+ref"),
                            (P.PFEM_SOLVE_F32_REFINED_FF, "f32+ff")):
            m = proj.p2m(v, shape=P.PFEM_SHAPE_QUADRATIC, solve=solve)
            code, _ = proj.status()
            assert code == 0
            got = m[J0:J1, :, 0].float().cpu().numpy().astype(np.float64)
            errs[(str(vt), name)] = float(np.abs(got - ref).max() / scale)
    print("precision study, max error / max|rho| vs FP64 oracle:", errs)
    for (vt, _), e in errs.items():
        assert e < (1e-6 if "float32" in vt else 1e-2), errs
