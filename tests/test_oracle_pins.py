"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it follows.  None of them re-types an oracle formula: they
check properties (moment identities, exact reproduction, empty circles, library
pseudo-inverse, convergence orders, invariances, adjoint identities, finite differences)
that a dropped term, a wrong sign or index, or a transposed operand would break.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from workloads import generators as G

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def offsets(pos, idx, n, I, J):
    """Minimal-image offsets of particles idx from node (I, J)."""
    nc = n - 1
    q = np.array([(I % nc) / nc, (J % nc) / nc])
    d = pos[idx] - q
    return d - np.rint(d)


@pytest.fixture(scope="module")
def tiny():
    pr = G.config_tiny()
    return pr, O.build_cells(pr.n, pr.pos)


# ------------------------------------------------------------------ cell list


def test_cell_list_matches_stable_sort(tiny):
    """Stable bin by mesh cell, ordered by (cell, original index)."""
    pr, cells = tiny
    nc = pr.n - 1
    q = O.fixed_point(pr.pos)
    cx = (q[:, 0].astype(np.uint64) * np.uint64(nc)) >> np.uint64(32)
    cy = (q[:, 1].astype(np.uint64) * np.uint64(nc)) >> np.uint64(32)
    cell = (cy * np.uint64(nc) + cx).astype(np.int64)
    perm = np.argsort(cell, kind="stable")
    assert np.array_equal(cells.perm, perm)
    counts = np.bincount(cell, minlength=nc * nc)
    assert np.array_equal(cells.cell_start, np.concatenate([[0], np.cumsum(counts)]))
    assert np.array_equal(cells.qs, q[perm])


# ------------------------------------------------------------------ Delaunay (App. B)


def _stars(cells, N):
    return [O.star(cells, m) for m in range(N)]


def _incircle_int(a, b, c, d):
    adx, ady = a[0] - d[0], a[1] - d[1]
    bdx, bdy = b[0] - d[0], b[1] - d[1]
    cdx, cdy = c[0] - d[0], c[1] - d[1]
    return ((adx * adx + ady * ady) * (bdx * cdy - bdy * cdx)
            + (bdx * bdx + bdy * bdy) * (cdx * ady - cdy * adx)
            + (cdx * cdx + cdy * cdy) * (adx * bdy - ady * bdx))


@pytest.mark.parametrize("jitter", [0.3, 0.0, "uniform"])
def test_delaunay_empty_circles_brute_force(jitter):
    """Every star triangle has an empty circumcircle (App. B, Delaunay definition), checked
    against all particles in exact integer arithmetic; an unjittered lattice (cocircular
    squares everywhere) only needs 'not strictly inside'.  Also on uniform random particles
    (no lattice: larger empty circles, star sizes from 3 to 11 here)."""
    M = 20
    if jitter == "uniform":
        pos = G.uniform01(G.SEED_BASE + 98, 2 * M * M).reshape(M * M, 2)
    else:
        pos = G.jittered_lattice(M, jitter, G.SEED_BASE + 99)
    pos = np.round(pos * 4096.0) / 4096.0 % 1.0          # exact small-integer coordinates
    X = np.round(pos * 4096.0).astype(np.int64)
    assert len({tuple(x) for x in X}) == len(X)           # no duplicates after rounding
    cells = O.build_cells(11, pos)
    N = M * M
    stars = _stars(cells, N)
    degs = np.array([len(s) for s in stars])
    assert degs.sum() == 6 * N                           # torus: E = 3N
    for v in range(N):
        s = stars[v]
        rel = X - X[v]
        rel = (rel + 2048) % 4096 - 2048                 # minimal image
        for k in range(len(s)):
            a, b = s[k], s[(k + 1) % len(s)]
            assert v in stars[a] and v in stars[b]
            A, B = rel[a], rel[b]
            assert A[0] * B[1] - A[1] * B[0] > 0         # CCW fan
            others = np.ones(N, bool)
            others[[v, a, b]] = False
            inc = _incircle_int(np.zeros(2, np.int64), A, B, rel[others].T)
            assert np.all(inc <= 0), (v, a, b)


def test_delaunay_matches_qhull(tiny):
    """Stars equal Qhull's Delaunay neighbours on the 3x3 periodic tiling (generic input)."""
    spatial = pytest.importorskip("scipy.spatial")
    M = 24
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 98)
    N = M * M
    tiles = np.concatenate([pos + [dx, dy] for dy in (-1, 0, 1) for dx in (-1, 0, 1)])
    tri = spatial.Delaunay(tiles)
    indptr, indices = tri.vertex_neighbor_vertices
    cells = O.build_cells(13, pos)
    centre = 4 * N
    for m in range(N):
        qh = set(int(j) % N for j in indices[indptr[centre + m]: indptr[centre + m + 1]])
        assert set(O.star(cells, m).tolist()) == qh, m


# ------------------------------------------------------------------ moment identities


def _moments(pos, idx, w, n, I, J):
    d = offsets(pos, idx, n, I, J)
    m0 = w.sum()
    m1 = (w[:, None] * d).sum(0)
    m2 = np.array([(w * d[:, 0] ** 2).sum(), (w * d[:, 0] * d[:, 1]).sum(), (w * d[:, 1] ** 2).sum()])
    return m0, m1, m2


def _some_nodes(n, count, seed):
    u = G.uniform01(seed, 2 * count)
    return [(int(u[2 * i] * n), int(u[2 * i + 1] * n)) for i in range(count)]


def test_linear_fe_moments(tiny):
    """Linear FE: partition of unity (C0), linear precision (C1), nonnegative barycentric
    weights, and quadratic precision fails (noC2)."""
    pr, cells = tiny
    h = 1.0 / pr.M
    worst2 = 0.0
    for I, J in _some_nodes(pr.n, 200, 7):
        idx, w, tri, _ = O.node_weights(cells, I, J, shape=0)
        assert len(idx) == 3 and set(idx) == set(tri)
        assert np.all(w >= -1e-15)
        m0, m1, m2 = _moments(pr.pos, idx, w, pr.n, I, J)
        assert abs(m0 - 1) < 1e-14
        assert np.abs(m1).max() < 1e-16 + 1e-14 * h
        worst2 = max(worst2, np.abs(m2).max())
    assert worst2 > 0.05 * h * h


def test_qcsf_moments(tiny):
    """QCSF: partition of unity, linear and quadratic precision (C0, C1, C2) at every node."""
    pr, cells = tiny
    h = 1.0 / pr.M
    for J in range(pr.n):
        for I in range(pr.n):
            idx, w, tri, rank = O.node_weights(cells, I, J, shape=1)
            assert rank == 6
            m0, m1, m2 = _moments(pr.pos, idx, w, pr.n, I, J)
            assert abs(m0 - 1) < 1e-13
            assert np.abs(m1).max() < 1e-13 * h
            assert np.abs(m2).max() < 1e-12 * h * h, (I, J, m2)


def test_edge_constraints_and_min_norm(tiny):
    """Per edge: eqs. (A0), (A1), (condquad) hold, and A is the minimum-norm solution
    (App. A), i.e. LAPACK's pseudo-inverse applied to the right-hand side."""
    pr, cells = tiny
    for I, J in _some_nodes(pr.n, 60, 11):
        tri, lam, edges, ranks = O.node_edges(cells, I, J)
        assert abs(lam.sum() - 1) < 1e-14 and np.all(lam >= -1e-15)
        for e, (S, A) in enumerate(edges):
            nu, sg = tri[e], tri[(e + 1) % 3]
            assert nu in S and sg in S and len(set(S.tolist())) == len(S) >= 6
            d = offsets(pr.pos, S, pr.n, I, J)
            dn = offsets(pr.pos, np.array([nu]), pr.n, I, J)[0]
            ds = offsets(pr.pos, np.array([sg]), pr.n, I, J)[0]
            scale = np.abs(d).max()
            assert abs(A.sum()) < 1e-12
            assert np.abs(A @ d).max() < 1e-12 * scale
            rhs = 0.5 * (np.outer(dn, ds) + np.outer(ds, dn) - np.outer(dn, dn) - np.outer(ds, ds))
            lhs = np.einsum("k,ki,kj->ij", A, d, d)
            assert np.abs(lhs - rhs).max() < 1e-12 * scale ** 2
            # eq. (A2_2): the same condition written translation-invariantly
            lhs2 = np.einsum("k,ki,kj->ij", A, d - dn, d - ds)
            assert np.abs(lhs2 + 0.5 * np.outer(dn - ds, dn - ds)).max() < 1e-12 * scale ** 2
            P = np.stack([np.ones(len(S)), d[:, 0], d[:, 1], d[:, 0] ** 2, d[:, 0] * d[:, 1],
                          d[:, 1] ** 2])
            b = np.array([0, 0, 0, rhs[0, 0], rhs[0, 1], rhs[1, 1]])
            A_ref = np.linalg.pinv(P) @ b
            assert np.abs(A - A_ref).max() < 1e-9 * max(1.0, np.abs(A_ref).max())


def test_rank_deficient_edge_is_the_pseudo_inverse_solution():
    """A rank-deficient edge system (App. A: SVD with rank detection).  In 2048^2 uniform
    random particles, node (245, 118) lies in a triangle with a 0.08-spacing edge whose
    stencil has five particles: six conditions, five unknowns, rank 5.  The oracle's A must
    be LAPACK's pseudo-inverse solution: the least-squares optimum (P^T (P A - b) = 0, the
    conditions cannot all hold) of minimum norm."""
    N = 2048 * 2048
    pos = G.uniform01(G.SEED_BASE + 62, 2 * N).reshape(N, 2)
    cells = O.build_cells(1025, pos)
    I, J = 245, 118
    tri, lam, edges, ranks = O.node_edges(cells, I, J)
    e = int(np.argmin(ranks))
    S, A = edges[e]
    assert ranks[e] == 5 and len(S) == 5
    nu, sg = tri[e], tri[(e + 1) % 3]
    d = offsets(pos, S, 1025, I, J)
    dn = offsets(pos, np.array([nu]), 1025, I, J)[0]
    ds = offsets(pos, np.array([sg]), 1025, I, J)[0]
    mid, L = 0.5 * (dn + ds), np.linalg.norm(dn - ds)
    x = (d - mid) / L                                  # the frame does not change A (eq. A2_2)
    t = (dn - ds) / L
    P = np.stack([np.ones(len(S)), x[:, 0], x[:, 1], x[:, 0] ** 2, x[:, 0] * x[:, 1], x[:, 1] ** 2])
    b = np.array([0, 0, 0, -0.5 * t[0] ** 2, -0.5 * t[0] * t[1], -0.5 * t[1] ** 2])
    A_ref = np.linalg.pinv(P) @ b
    assert np.abs(A - A_ref).max() < 1e-9 * max(1.0, np.abs(A_ref).max())
    assert np.abs(P.T @ (P @ A - b)).max() < 1e-12
    assert np.abs(P @ A - b).max() > 1e-6               # inconsistent: least squares, not exact


def test_interpolating_property(tiny):
    """A node that coincides with a particle takes that particle's value (App. B: the
    extended functions stay interpolating)."""
    pr, _ = tiny
    pos = pr.pos.copy()
    nc = pr.n - 1
    I0, J0 = 9, 21
    mu = int(np.argmin(np.sum((pos - [I0 / nc, J0 / nc]) ** 2, axis=1)))
    pos[mu] = [I0 / nc, J0 / nc]
    for shape in (0, 1):
        mesh = O.p2m(pr.n, pos, pr.vals, shape=shape)
        assert np.abs(mesh[J0, I0] - pr.vals[mu]).max() < 1e-14


def test_negative_lobes_and_overshoot():
    """QCSF weights can be negative and the slotted-disk indicator overshoots 1 and goes
    below 0, while linear FE stays a convex combination (Sec. 3.1 discussion of Gibbs
    effects; eq. A0)."""
    gold = json.load(open(os.path.join(GOLDEN, "zalesak_overshoot.json")))
    n, M = 65, 128
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 21)
    ind = G.zalesak_disk(pos)[:, None]
    mq = O.p2m(n, pos, ind, shape=1, nthreads=4)
    ml = O.p2m(n, pos, ind, shape=0, nthreads=4)
    assert (mq.max() > 1.0 + 1e-3) == gold["quadratic_indicator_exceeds_one"]
    assert mq.min() < -1e-3
    assert (ml.min() >= -1e-15 and ml.max() <= 1 + 1e-15) == gold["linear_indicator_within_0_1"]
    cells = O.build_cells(n, pos)
    negs = sum((O.node_weights(cells, I, J, 1)[1] < 0).any() for I, J in _some_nodes(n, 20, 3))
    assert (negs > 0) == gold["quadratic_has_negative_weights"]


# ------------------------------------------------------------------ convergence orders


def _slope(hs, errs):
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


def test_projection_orders():
    """Under refinement at fixed h/H = 1/2 on Taylor-Green fields, P2M errors fall as h^2
    (linear FE) and h^3 (QCSF), M2P errors as H^2 (Sec. 2.1)."""
    gold = json.load(open(os.path.join(GOLDEN, "projection_orders.json")))
    hs, el, eq, em = [], [], [], []
    for nc in (16, 32, 64, 128):
        n, M = nc + 1, 2 * nc
        pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 40 + nc)
        vals = G.taylor_green(pos)
        nodes = np.stack(np.meshgrid(np.arange(n) / nc, np.arange(n) / nc), -1).reshape(-1, 2)
        exact = G.taylor_green(nodes).reshape(n, n, 3)
        rel = lambda m: np.sqrt(((m - exact) ** 2).sum() / (exact ** 2).sum())  # eq. L2_error
        el.append(rel(O.p2m(n, pos, vals, shape=0, nthreads=8)))
        eq.append(rel(O.p2m(n, pos, vals, shape=1, nthreads=8)))
        back = O.m2p(n, pos, exact)
        em.append(np.sqrt(((back - vals) ** 2).sum() / (vals ** 2).sum()))
        hs.append(1.0 / M)
    sl, sq, sm = _slope(hs, el), _slope(hs, eq), _slope(hs, em)
    assert abs(sl - gold["p2m_linear_order"]) < 0.3, sl
    assert abs(sq - gold["p2m_quadratic_order"]) < 0.35, sq
    assert abs(sm - gold["m2p_linear_order"]) < 0.3, sm


def test_m2p_reproduces_linear_fields():
    """Linear FE on the mesh reproduces any linear field exactly (eq. m2p with FE)."""
    n, M = 17, 40
    nc = n - 1
    pos = G.jittered_lattice(M, 0.3, G.SEED_BASE + 50)
    II, JJ = np.meshgrid(np.arange(n), np.arange(n))
    mesh = np.stack([0.3 + 1.7 * II - 0.4 * JJ, -2 + 0.5 * II + 3 * JJ], -1).astype(float)
    out = O.m2p(n, pos, mesh)
    q = O.fixed_point(pos)
    i = ((q[:, 0].astype(np.uint64) * np.uint64(nc)) >> np.uint64(32)).astype(np.int64)
    j = ((q[:, 1].astype(np.uint64) * np.uint64(nc)) >> np.uint64(32)).astype(np.int64)
    s = (pos[:, 0] - i / nc - np.rint(pos[:, 0] - i / nc)) * nc + i
    t = (pos[:, 1] - j / nc - np.rint(pos[:, 1] - j / nc)) * nc + j
    expect = np.stack([0.3 + 1.7 * s - 0.4 * t, -2 + 0.5 * s + 3 * t], -1)
    assert np.abs(out - expect).max() < 1e-12


# ------------------------------------------------------------------ invariances


def test_translation_and_rotation_invariance():
    """The construction is translation and rotation invariant (eq. A2_2): shifting all
    particles by one mesh spacing shifts P2M by one node; a quarter turn of the torus turns
    the P2M field."""
    n, M = 33, 64
    nc = n - 1
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 60)
    pos = np.round(pos * 2.0 ** 32) / 2.0 ** 32 % 1.0
    vals = G.taylor_green(pos)
    base = O.p2m(n, pos, vals, shape=1, nthreads=8)
    sh = (pos + [1.0 / nc, 0.0]) % 1.0
    shifted = O.p2m(n, sh, vals, shape=1, nthreads=8)
    assert np.abs(shifted[:, 1:] - base[:, :-1]).max() < 1e-12
    rot = np.stack([(1.0 - pos[:, 1]) % 1.0, pos[:, 0]], -1)
    rotated = O.p2m(n, rot, vals, shape=1, nthreads=8)
    # node (I, J) -> ((nc - J) mod nc, I)
    for J in range(nc):
        for I in range(nc):
            assert np.abs(rotated[I, (nc - J) % nc] - base[J, I]).max() < 1e-12


def test_duplicate_particles_rejected():
    pos = G.jittered_lattice(16, 0.25, 5)
    pos[7] = pos[3]
    with pytest.raises(O.OracleError) as e:
        O.p2m(9, pos, np.ones((pos.shape[0], 1)), shape=1)
    assert e.value.code == 5


# ------------------------------------------------------------------ adjoints


@pytest.fixture(scope="module")
def small():
    n, M = 17, 32
    pos = G.jittered_lattice(M, 0.25, G.SEED_BASE + 70)
    vals = G.taylor_green(pos)[:, :2].copy()
    g = np.random.default_rng(1).standard_normal((n, n, 2))
    return n, pos, vals, g


@pytest.mark.parametrize("shape", [0, 1])
def test_p2m_adjoint_values_dot_product(small, shape):
    """<P2M a, g> = <a, P2M^T g> (the value adjoint is the transposed weights)."""
    n, pos, vals, g = small
    a = np.random.default_rng(2).standard_normal(vals.shape)
    gv, _ = O.p2m_backward(n, pos, a, g, shape=shape)
    lhs = (O.p2m(n, pos, a, shape=shape) * g).sum()
    assert abs(lhs - (a * gv).sum()) < 1e-12 * abs(lhs)


def _same_topology(n, p1, p2, shape):
    c1, c2 = O.build_cells(n, p1), O.build_cells(n, p2)
    for J in range(n):
        for I in range(n):
            a = O.node_weights(c1, I, J, shape)[0]
            b = O.node_weights(c2, I, J, shape)[0]
            if sorted(a.tolist()) != sorted(b.tolist()):
                return False
    return True


@pytest.mark.parametrize("shape", [0, 1])
def test_p2m_position_gradient_vs_central_differences(small, shape):
    """Complex-step position gradient vs central differences (step 1e-6, FP64)."""
    n, pos, vals, g = small
    _, gp = O.p2m_backward(n, pos, vals, g, shape=shape)
    rng = np.random.default_rng(3)
    checked = 0
    for m in rng.choice(pos.shape[0], 12, replace=False):
        for dim in (0, 1):
            step = 1e-6
            pp, pm = pos.copy(), pos.copy()
            pp[m, dim] += step
            pm[m, dim] -= step
            if not _same_topology(n, pp, pm, shape):
                continue
            fd = ((O.p2m(n, pp, vals, shape) * g).sum() - (O.p2m(n, pm, vals, shape) * g).sum()) / (2 * step)
            assert abs(fd - gp[m, dim]) < 1e-6 * max(1.0, abs(fd)), (m, dim, fd, gp[m, dim])
            checked += 1
    assert checked >= 16


@pytest.mark.parametrize("shape", [0, 1])
def test_node_weight_derivatives_vs_central_differences(small, shape):
    """The complex-step derivative of one node's weights with respect to one particle
    coordinate equals the central difference of the weights themselves (step 1e-6, FP64) for
    every particle of the node's weight set, when the perturbation leaves the topology alone.
    A wrong sign or a dropped chain-rule term in the complex-step path would fail this."""
    n, pos, _, _ = small
    cells = O.build_cells(n, pos)
    rng = np.random.default_rng(17)
    checked = 0
    for node in rng.choice(n * n, 10, replace=False):
        J, I = divmod(int(node), n)
        idx, w, _, _ = O.node_weights(cells, I, J, shape)
        for m in rng.choice(idx, 2, replace=False):
            for dim in (0, 1):
                didx, dw = O.node_weight_derivs(cells, I, J, int(m), dim, shape)
                assert np.array_equal(didx, idx)
                step = 1e-6
                pp, pm = pos.copy(), pos.copy()
                pp[m, dim] += step
                pm[m, dim] -= step
                ip, wp, _, _ = O.node_weights(O.build_cells(n, pp), I, J, shape)
                im, wm, _, _ = O.node_weights(O.build_cells(n, pm), I, J, shape)
                if sorted(ip) != sorted(idx) or sorted(im) != sorted(idx):
                    continue
                fp = dict(zip(ip.tolist(), wp)); fm = dict(zip(im.tolist(), wm))
                fd = np.array([(fp[k] - fm[k]) / (2 * step) for k in idx.tolist()])
                assert np.abs(fd - dw).max() <= 1e-6 * max(1.0, np.abs(fd).max()), (I, J, m, dim)
                checked += 1
    assert checked >= 20


def test_rank_deficient_node_derivatives_vs_central_differences():
    """512^2 uniform random particles on the 257^2 mesh: node (68, 52) has an edge whose
    stencil is five particles, so its system is inconsistent and the oracle's forward takes the
    least-squares pseudo-inverse solution by SVD (App. A), which depends on the edge frame.  The
    complex-step derivative (normal equations of the five-column system, frame differentiated)
    matches central differences of the SVD forward (step 1e-7) for every particle of the node's
    weight set in both coordinates."""
    n, M = 257, 512
    pos = G.uniform01(G.SEED_BASE + 62, 2 * M * M).reshape(M * M, 2)
    cells = O.build_cells(n, pos)
    I, J = 68, 52
    idx, w, _, rank = O.node_weights(cells, I, J, 1)
    assert rank == 5
    checked = 0
    for m in idx.tolist():
        for dim in (0, 1):
            didx, dw = O.node_weight_derivs(cells, I, J, m, dim, 1)
            step = 1e-7
            pp, pm = pos.copy(), pos.copy()
            pp[m, dim] += step
            pm[m, dim] -= step
            ip, wp, _, rp = O.node_weights(O.build_cells(n, pp), I, J, 1)
            im, wm, _, rm = O.node_weights(O.build_cells(n, pm), I, J, 1)
            assert sorted(ip) == sorted(idx) and sorted(im) == sorted(idx) and rp == rm == 5
            fp = dict(zip(ip.tolist(), wp)); fm = dict(zip(im.tolist(), wm))
            fd = np.array([(fp[k] - fm[k]) / (2 * step) for k in idx.tolist()])
            assert np.abs(fd - dw).max() <= 1e-5 * max(1.0, np.abs(fd).max()), (m, dim)
            checked += 1
    assert checked == 2 * len(idx)


def test_m2p_adjoint(small):
    """M2P: <M2P f, g> = <f, M2P^T g>, and the position gradient vs central differences."""
    n, pos, vals, _ = small
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n, n, 2))
    gv = rng.standard_normal((pos.shape[0], 2))
    gm, gp = O.m2p_backward(n, pos, f, gv)
    lhs = (O.m2p(n, pos, f) * gv).sum()
    assert abs(lhs - (f * gm).sum()) < 1e-12 * abs(lhs)
    for m in rng.choice(pos.shape[0], 10, replace=False):
        for dim in (0, 1):
            step = 1e-7
            pp, pm = pos.copy(), pos.copy()
            pp[m, dim] += step
            pm[m, dim] -= step
            fd = ((O.m2p(n, pp, f) - O.m2p(n, pm, f)) * gv).sum() / (2 * step)
            assert abs(fd - gp[m, dim]) < 1e-6 * max(1.0, abs(fd))


def test_node_range_is_validated():
    pos = G.jittered_lattice(16, 0.25, 5)
    with pytest.raises(O.OracleError) as e:
        O.p2m(9, pos, np.ones((pos.shape[0], 1)), shape=1, node_range=(-5, 10))
    assert e.value.code == 1


# ------------------------------------------------------------------ mesh QCSF (M2P)


def test_mesh_edge_coefficients():
    """Mesh-edge coefficients satisfy eqs. A0, A1, condquad on their 10-node stencils and are
    the minimum-norm solution (LAPACK pseudo-inverse)."""
    for t, d in enumerate(((1, 0), (0, 1), (1, 1))):
        off, A = O.mesh_edge(t)
        assert len(off) == 10 and len({tuple(o) for o in off}) == 10
        d = np.array(d, float)
        x = off.astype(float)
        assert abs(A.sum()) < 1e-13 and np.abs(A @ x).max() < 1e-13
        rhs = 0.5 * (-np.outer(d, d))          # nodes (0,0) and d: eq. condquad
        lhs = np.einsum("k,ki,kj->ij", A, x, x)
        assert np.abs(lhs - rhs).max() < 1e-13
        P = np.stack([np.ones(10), x[:, 0], x[:, 1], x[:, 0] ** 2, x[:, 0] * x[:, 1], x[:, 1] ** 2])
        b = np.array([0, 0, 0, rhs[0, 0], rhs[0, 1], rhs[1, 1]])
        assert np.abs(A - np.linalg.pinv(P) @ b).max() < 1e-12


def test_mesh_qcsf_m2p_reproduces_quadratics():
    """Mesh QCSF reproduce quadratic fields exactly (eq. C2), where linear FE do not; checked
    away from the periodic seam with a non-periodic quadratic in node coordinates."""
    n = 33
    nc = n - 1
    II, JJ = np.meshgrid(np.arange(n), np.arange(n))
    quad = lambda X, Y: 0.7 + 0.3 * X - 0.2 * Y + 0.05 * X * X - 0.03 * X * Y + 0.02 * Y * Y
    mesh = quad(II.astype(float), JJ.astype(float))[..., None]
    rng = np.random.default_rng(0)
    pos = rng.uniform(3.0 / nc, (nc - 4.0) / nc, size=(500, 2))
    exact = quad(pos[:, 0] * nc, pos[:, 1] * nc)
    q = O.m2p_quadratic(n, pos, mesh)[:, 0]
    l = O.m2p(n, pos, mesh)[:, 0]
    assert np.abs(q - exact).max() < 1e-12 * np.abs(exact).max()
    assert np.abs(l - exact).max() > 1e-4
    # constants and linear fields everywhere (partition of unity, linear precision)
    ones = np.ones((n, n, 1))
    assert np.abs(O.m2p_quadratic(n, pos, ones) - 1).max() < 1e-13


def test_mesh_qcsf_m2p_order_and_interpolation():
    """M2P error on Taylor-Green fields falls as H^3 with mesh QCSF (H^2 with linear FE), and
    a particle on a node takes the node's value."""
    errs_q, errs_l, hs = [], [], []
    for nc in (16, 32, 64, 128):
        n = nc + 1
        pos = G.jittered_lattice(2 * nc, 0.25, G.SEED_BASE + 80 + nc)
        nodes = np.stack(np.meshgrid(np.arange(n) / nc, np.arange(n) / nc), -1).reshape(-1, 2)
        mesh = G.taylor_green(nodes).reshape(n, n, 3)
        exact = G.taylor_green(pos)
        rel = lambda v: np.sqrt(((v - exact) ** 2).sum() / (exact ** 2).sum())
        errs_q.append(rel(O.m2p_quadratic(n, pos, mesh)))
        errs_l.append(rel(O.m2p(n, pos, mesh)))
        hs.append(1.0 / nc)
    sq = np.polyfit(np.log(hs), np.log(errs_q), 1)[0]
    sl = np.polyfit(np.log(hs), np.log(errs_l), 1)[0]
    assert abs(sl - 2) < 0.3 and abs(sq - 3) < 0.35, (sl, sq)
    n = 17
    mesh = np.random.default_rng(2).standard_normal((n, n, 2))
    mesh[-1] = mesh[0]
    mesh[:, -1] = mesh[:, 0]
    p = np.array([[5 / 16, 9 / 16]])
    assert np.abs(O.m2p_quadratic(n, p, mesh)[0] - mesh[9, 5]).max() < 1e-14


# ------------------------------------------------------------------ the projection loop's move


def test_midpoint_move_of_a_uniform_field_is_a_translation():
    """A uniform mesh velocity is reproduced exactly by linear FE (eq. C1), so the midpoint
    step is the exact translation r + dt u (Sec. 3.2 scheme), wrapped into the torus."""
    n = 33
    pos = G.uniform01(G.SEED_BASE + 500, 2000).reshape(1000, 2)
    vel = np.zeros((n, n, 2))
    vel[..., 0], vel[..., 1] = 0.37, -1.9
    new = O.advect_midpoint(n, pos, vel, 0.05)
    want = pos + 0.05 * np.array([0.37, -1.9])
    want -= np.floor(want)
    d = new - want
    assert np.abs(d - np.rint(d)).max() < 1e-14


def test_midpoint_move_of_a_rotation_is_second_order_taylor():
    """Rigid rotation about the centre sampled at the nodes: away from the periodic seam the
    field is linear, which linear FE reproduces exactly, so one midpoint step maps
    r - c -> (I + dt A + (dt A)^2 / 2)(r - c) with A = omega [[0, -1], [1, 0]] (the midpoint
    scheme's second-order Taylor map for a linear field).  A full step in place of the half step
    would break this."""
    n, om, dt = 65, 2 * np.pi, 0.01
    g = np.arange(n) / (n - 1)
    X, Y = np.meshgrid(g, g)
    vel = np.stack([-om * (Y - 0.5), om * (X - 0.5)], -1)
    pos = 0.2 + 0.6 * G.uniform01(G.SEED_BASE + 501, 4000).reshape(2000, 2)
    new = O.advect_midpoint(n, pos, vel, dt)
    A = om * np.array([[0.0, -1.0], [1.0, 0.0]])
    T = np.eye(2) + dt * A + 0.5 * (dt * A) @ (dt * A)
    want = 0.5 + (pos - 0.5) @ T.T
    assert np.abs(new - want).max() < 1e-13
