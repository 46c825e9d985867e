// backward.cu -- adjoint of P2M with respect to particle values and positions (no paper
// counterpart; the paper only runs the forward projection).
//
// Forward, per node i:  alpha_i = sum_mu w_{i mu}(r) alpha_mu  with
//   w_{i mu} = lambda_mu [mu in T] + sum_{e=(nu,sg) in T} c_e A_{mu e},   c_e = 2 lambda_nu lambda_sg,
//   A_{mu e} = p_mu . y_e,  M_e y_e = b_e,  M_e = sum_{mu in S_e} p_mu p_mu^T.
// With beta_mu = gbar_i . alpha_mu, the node contributes
//   dL/dalpha_mu += w_{i mu} gbar_i,
//   dL/dr via lambda (barycentric cofactors) and via every edge: u = sum beta_mu p_mu,
//   B_e = u . y_e, z = M_e^{-1} u (one extra solve), and for each stencil member
//   pbar_mu = c_e [(beta_mu - z.p_mu) y_e - (y_e.p_mu) z],  tbar from b_e, lambdabar from c_e B_e.
// The frame (edge midpoint, edge length) is held fixed: A does not depend on it (eq. A2_2), so
// the derivative at a fixed frame is the derivative of A.
//
// Determinism without atomics on values: phase 1 writes each node's entries (slot, w, dpos)
// into [n*n, K] arrays; phase 2 builds a transposed index by a stable counting sort keyed by
// particle slot (entries per particle ordered by entry id) and gathers per particle.
#include <algorithm>

#include "internal.h"
#include "p2m.cuh"

namespace pfem {

struct BwdArgs {
    P2MArgs f;                  // forward geometry/values (f.out unused)
    const void *grad_mesh;      // [n*n, C]
    int K;                      // entries per node
    int *e_slot;                // [n*n*K]
    void *e_w;                  // [n*n*K] R
    void *e_dpos;               // [n*n*K*2] R (may be null: value gradient only)
};

constexpr int KBWD = 32;   // distinct particles per node kept by the recompute kernel

// The adjoint of one node over its particle set (us[0..nu), stencil masks vm, tri[e] = us[vi[e]]):
// uw the weights, ub = gbar . alpha per particle, udx/udy the position adjoints (all zero on
// entry).  Returns 0, or -PFEM_DEFER when a moment matrix is below the forward's fast-solve
// tolerance: the node goes to the adjoint's fix pass, as the forward sends it to its own.
template <typename P, typename V, typename R, typename S, int SHAPE, bool POS>
__device__ __forceinline__ int bwd_u_solve(const BwdArgs &b, const NodePos<P, R> &np, const R g[8],
                                           const int tri[3], const int *us, int nu,
                                           const unsigned vm[3], const int vi[3], R *uw, R *ub,
                                           R *udx, R *udy)
{
    const P2MArgs &a = b.f;
    int st = 0;
    for (int i = 0; i < nu; ++i) {
        R v[8];
        load_vals<V, R>((const V *)a.vals, a.perm, us[i], a.C, v);
        R t = R(0);
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < a.C) t = fma(g[c], v[c], t);
        ub[i] = t;
    }
    R d[3][2];
#pragma unroll
    for (int e = 0; e < 3; ++e) np.off(a.pos, tri[e], d[e][0], d[e][1]);
    const R Na = d[1][0] * d[2][1] - d[1][1] * d[2][0];
    const R Nb = d[2][0] * d[0][1] - d[2][1] * d[0][0];
    const R Nc = d[0][0] * d[1][1] - d[0][1] * d[1][0];
    const R A2 = Na + Nb + Nc;
    const R lam[3] = {Na / A2, Nb / A2, Nc / A2};
    R lbar[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        uw[vi[e]] += lam[e];
        lbar[e] = ub[vi[e]];
    }
    auto offset = [&](int i, S &x, S &y) {
        R dx, dy;
        np.off(a.pos, us[i], dx, dy);
        x = S(dx);
        y = S(dy);
    };
    if (SHAPE == PFEM_SHAPE_QUADRATIC)
        for (int e = 0; e < 3 && st == 0; ++e) {
            const int f = e == 2 ? 0 : e + 1;
            const unsigned mask = vm[e] | vm[f];
            const S rnx = S(d[e][0]), rny = S(d[e][1]), rsx = S(d[f][0]), rsy = S(d[f][1]);
            const S mx = (rnx + rsx) * S(0.5), my = (rny + rsy) * S(0.5);
            const S ex = rnx - rsx, ey = rny - rsy;
            const S inv = S(1) / sqrt(ex * ex + ey * ey);
            Moment<S> M;
            M.zero();
            S u[6] = {S(0), S(0), S(0), S(0), S(0), S(0)};
            for (unsigned m = mask; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                S ox, oy;
                offset(i, ox, oy);
                const S x = (ox - mx) * inv, y = (oy - my) * inv;
                M.add(x, y);
                const S bt = S(ub[i]);
                const S p[6] = {S(1), x, y, x * x, x * y, y * y};
#pragma unroll
                for (int r = 0; r < 6; ++r) u[r] = fma(bt, p[r], u[r]);
            }
            if (!M.factor(FastTol<S>::v)) { st = -PFEM_DEFER; break; }
            const S tx = ex * inv, ty = ey * inv;
            const S bb[6] = {S(0), S(0), S(0), S(-0.5) * tx * tx, S(-0.5) * tx * ty,
                             S(-0.5) * ty * ty};
            S y[6], z[6];
            M.solve(bb, y);
            M.solve(u, z);
            const S ce = S(2) * S(lam[e]) * S(lam[f]);
            S Be = S(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) Be = fma(u[r], y[r], Be);
            lbar[e] += R(S(2) * S(lam[f]) * Be);
            lbar[f] += R(S(2) * S(lam[e]) * Be);
            for (unsigned m = mask; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                S ox, oy;
                offset(i, ox, oy);
                const S x = (ox - mx) * inv, yy = (oy - my) * inv;
                const S p[6] = {S(1), x, yy, x * x, x * yy, yy * yy};
                S Am = S(0), Zm = S(0);
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    Am = fma(p[r], y[r], Am);
                    Zm = fma(p[r], z[r], Zm);
                }
                uw[i] += R(ce * Am);
                if (POS) {
                    const S bt = S(ub[i]);
                    S pb[6];
#pragma unroll
                    for (int r = 0; r < 6; ++r) pb[r] = ce * ((bt - Zm) * y[r] - Am * z[r]);
                    const S xb = pb[1] + S(2) * x * pb[3] + yy * pb[4];
                    const S yb = pb[2] + x * pb[4] + S(2) * yy * pb[5];
                    udx[i] += R(xb * inv);
                    udy[i] += R(yb * inv);
                }
            }
            if (POS) {
                // b = [0,0,0,-tx^2/2,-tx ty/2,-ty^2/2], t = (r_nu - r_sg)/s
                const S txb = ce * (-tx * z[3] - S(0.5) * ty * z[4]);
                const S tyb = ce * (-S(0.5) * tx * z[4] - ty * z[5]);
                udx[vi[e]] += R(txb * inv);
                udy[vi[e]] += R(tyb * inv);
                udx[vi[f]] -= R(txb * inv);
                udy[vi[f]] -= R(tyb * inv);
            }
        }
    if (POS && st == 0) {
        // lambda_k = N_k / A2 with N_a = d_b x d_c, N_b = d_c x d_a, N_c = d_a x d_b
        const R Lam = lbar[0] * lam[0] + lbar[1] * lam[1] + lbar[2] * lam[2];
        const R nb0 = (lbar[0] - Lam) / A2, nb1 = (lbar[1] - Lam) / A2, nb2 = (lbar[2] - Lam) / A2;
        // cross(u, v): d/du = (v.y, -v.x), d/dv = (-u.y, u.x)
        R gx[3] = {R(0), R(0), R(0)}, gy[3] = {R(0), R(0), R(0)};
        gx[1] += nb0 * d[2][1];  gy[1] -= nb0 * d[2][0];
        gx[2] -= nb0 * d[1][1];  gy[2] += nb0 * d[1][0];
        gx[2] += nb1 * d[0][1];  gy[2] -= nb1 * d[0][0];
        gx[0] -= nb1 * d[2][1];  gy[0] += nb1 * d[2][0];
        gx[0] += nb2 * d[1][1];  gy[0] -= nb2 * d[1][0];
        gx[1] -= nb2 * d[0][1];  gy[1] += nb2 * d[0][0];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            udx[vi[e]] += gx[e];
            udy[vi[e]] += gy[e];
        }
    }
    return st;
}

template <typename P, typename V, typename R, typename S, int SHAPE, bool POS>
__device__ __forceinline__ void bwd_node(const BwdArgs &b, int I, int J)
{
    const P2MArgs &a = b.f;
    const int nc = a.n - 1;
    const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
    const long long node = (long long)J * a.n + I;
    int *oslot = b.e_slot + node * b.K;
    R *ow = (R *)b.e_w + node * b.K;
    R *od = POS ? (R *)b.e_dpos + node * b.K * 2 : nullptr;

    R g[8];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        g[c] = c < a.C ? load_val<V, R>((const V *)b.grad_mesh + node * a.C + c) : R(0);
        any |= g[c] != R(0);
    }
    // the node's distinct particles U: slot, weight, beta = gbar . alpha, position adjoint
    int us[UMAX];
    R uw[UMAX], ub[UMAX], udx[UMAX], udy[UMAX];
    int nu = 0;
    int st = 0;
    if (any) {
        const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
        int tri[3];
        int stars[3][KMAX];
        int ns[3] = {0, 0, 0};
        st = locate(a.B, qn, a.R0, tri, stars[0], ns[0]);
        if (SHAPE == PFEM_SHAPE_QUADRATIC && st == 0)
            for (int e = 0; e < 3 && st == 0; ++e)
                if (ns[e] == 0) {
                    const int c = star_of(a.B, tri[e], a.R0, stars[e]);
                    if (c < 0) st = c;
                    else ns[e] = c;
                }
        if (st == 0) {
            NodePos<P, R> np;
            np.init(Iu, Ju, nc);
            bool over = false;
            auto add = [&](int s) -> int {
                for (int i = 0; i < nu; ++i)
                    if (us[i] == s) return i;
                if (nu == UMAX || nu == b.K) { over = true; return 0; }
                us[nu] = s;
                uw[nu] = udx[nu] = udy[nu] = R(0);
                return nu++;
            };
            int vi[3];
            unsigned vm[3] = {0u, 0u, 0u};
#pragma unroll
            for (int e = 0; e < 3; ++e) vi[e] = add(tri[e]);
            if (SHAPE == PFEM_SHAPE_QUADRATIC)
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    unsigned m = 1u << vi[e];
                    for (int i = 0; i < ns[e]; ++i) m |= 1u << add(stars[e][i]);
                    vm[e] = m;
                }
            if (over) st = -PFEM_DEFER;
            if (st == 0)
                st = bwd_u_solve<P, V, R, S, SHAPE, POS>(b, np, g, tri, us, nu, vm, vi, uw, ub,
                                                         udx, udy);
        }
        if (st != 0) {
            st = defer_or_error(a, st, node);
            if (st < 0) record_error(a.status, -st, node);
            nu = 0;
        }
    }
    for (int k = 0; k < b.K; ++k) {
        const bool v = k < nu;
        oslot[k] = v ? us[k] : -1;
        ow[k] = v ? uw[k] : R(0);
        if (POS) {
            od[2 * k] = v ? udx[k] : R(0);
            od[2 * k + 1] = v ? udy[k] : R(0);
        }
    }
}

template <typename P, typename V, typename R, typename S, int SHAPE, bool POS>
__global__ void __launch_bounds__(128, PFEM_P2M_MIN_BLOCKS) k_bwd_node(BwdArgs b)
{
    const int I = blockIdx.x * 16 + (threadIdx.x & 15);
    const int J = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (I >= b.f.n || J >= b.f.n) return;
    bwd_node<P, V, R, S, SHAPE, POS>(b, I, J);
}

// The adjoint with FP32 solves as two kernels, as in the forward: k_p2m_geom writes each
// node's record (particle set, stencil masks), this kernel solves the adjoint of the three edge
// systems with its own register budget and writes the node's entries.
template <typename P, typename V, typename R, typename S, bool POS>
__global__ void __launch_bounds__(128, 4) k_bwd_solve(BwdArgs b, NodeRecs r)
{
    const P2MArgs &a = b.f;
    const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= r.nodes) return;
    int *oslot = b.e_slot + node * b.K;
    R *ow = (R *)b.e_w + node * b.K;
    R *od = POS ? (R *)b.e_dpos + node * b.K * 2 : nullptr;
    R g[8];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        g[c] = c < a.C ? load_val<V, R>((const V *)b.grad_mesh + node * a.C + c) : R(0);
        any |= g[c] != R(0);
    }
    int us[UMAX];
    R uw[UMAX], ub[UMAX], udx[UMAX], udy[UMAX];
    int nu = 0;
    const int meta = r.meta[node];
    if (any && meta >= 0) {
        nu = meta & 31;
        const int vi[3] = {(meta >> 5) & 31, (meta >> 10) & 31, (meta >> 15) & 31};
        if (nu > b.K) {
            record_error(a.status, PFEM_ERR_CAPACITY, node);
            nu = 0;
        } else {
            for (int i = 0; i < nu; ++i) {
                us[i] = r.us[i * r.nodes + node];
                uw[i] = udx[i] = udy[i] = R(0);
            }
            unsigned vm[3];
            int tri[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                vm[e] = r.mask[e * r.nodes + node];
                tri[e] = us[vi[e]];
            }
            const int nc = a.n - 1;
            const int I = (int)(node % a.n), J = (int)(node / a.n);
            NodePos<P, R> np;
            np.init(I == nc ? 0 : I, J == nc ? 0 : J, nc);
            int st = bwd_u_solve<P, V, R, S, PFEM_SHAPE_QUADRATIC, POS>(
                b, np, g, tri, us, nu, vm, vi, uw, ub, udx, udy);
            if (st != 0) {
                st = defer_or_error(a, st, node);
                if (st < 0) record_error(a.status, -st, node);
                nu = 0;
            }
        }
    }
    for (int k = 0; k < b.K; ++k) {
        const bool v = k < nu;
        oslot[k] = v ? us[k] : -1;
        ow[k] = v ? uw[k] : R(0);
        if (POS) {
            od[2 * k] = v ? udx[k] : R(0);
            od[2 * k + 1] = v ? udy[k] : R(0);
        }
    }
}

// ---------------------------------------------------------------- fix pass
// The nodes the fast adjoint queued (an edge system below the forward's fast-solve tolerance,
// more particles than the fast pass holds, or a search that ran out of its region), recomputed
// in FP64 with the forward fix pass's geometry (widest search radius) and SVD solve.  For each
// edge, with P the 6 x k monomial matrix (the stencil in the edge frame), A = P^+ b its
// pseudo-inverse solution and Abar = c_e beta, the reverse-mode derivative of the pseudo-inverse
// at constant rank (Golub & Pereyra 1973) gives
//   Pbar = -u A^T + r (P^+ u)^T + z ((I - P^+ P) Abar)^T,   bbar = u,
// with u = P^+T Abar, z = P^+T A and r = b - P A (zero unless the system is inconsistent, as
// for a stencil of five particles).  A least-squares solution depends on the edge frame, so the
// frame's dependence on the edge endpoints (midpoint m, length s) is differentiated too.

// One edge.  pt: the k members' monomial rows (overwritten), x/y their frame coordinates,
// beta their gbar . alpha, b, ce = 2 lambda_nu lambda_sg.  Out: A (coefficients), xb/yb the
// adjoints of the members' frame coordinates, bb the adjoint of b, and Be = sum beta A.
static __device__ __noinline__ void edge_adjoint_svd(int k, double (*pt)[6], const double *x,
                                                     const double *y, const double *beta,
                                                     const double b[6], double ce, double *A,
                                                     double *xb, double *yb, double bb[6],
                                                     double &Be)
{
    double V[6][6], sig2[6];
    jacobi_svd(k, pt, V, sig2);
    const double thr2 = svd_threshold2(k, sig2);
    double vb[6], wA[6], wAA[6];
    for (int j = 0; j < 6; ++j) {
        double d = 0.0;
        for (int r = 0; r < 6; ++r) d = fma(V[r][j], b[r], d);
        vb[j] = sig2[j] > thr2 ? d : 0.0;
    }
    Be = 0.0;
    for (int i = 0; i < k; ++i) {
        double a = 0.0;
        for (int j = 0; j < 6; ++j)
            if (sig2[j] > thr2) a = fma(vb[j] / sig2[j], pt[i][j], a);
        A[i] = a;
        Be = fma(beta[i], a, Be);
    }
    for (int j = 0; j < 6; ++j) {
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < k; ++i) {
            s1 = fma(pt[i][j], ce * beta[i], s1);
            s2 = fma(pt[i][j], A[i], s2);
        }
        wA[j] = sig2[j] > thr2 ? s1 / sig2[j] : 0.0;    // (w_j . Abar) / sigma_j^2
        wAA[j] = sig2[j] > thr2 ? s2 / sig2[j] : 0.0;   // (w_j . A) / sigma_j^2
    }
    double u[6], z[6], r[6];
    for (int q = 0; q < 6; ++q) {
        double su = 0.0, sz = 0.0, sr = b[q];
        for (int j = 0; j < 6; ++j) {
            su = fma(V[q][j], wA[j], su);
            sz = fma(V[q][j], wAA[j], sz);
            sr = fma(-V[q][j], vb[j], sr);
        }
        u[q] = su;
        z[q] = sz;
        r[q] = sr;
        bb[q] = su;
    }
    for (int i = 0; i < k; ++i) {
        double pu = 0.0, pp = 0.0;
        for (int j = 0; j < 6; ++j)
            if (sig2[j] > thr2) {
                pu = fma(pt[i][j], wA[j] / sig2[j], pu);
                pp = fma(pt[i][j], wA[j], pp);
            }
        const double qi = ce * beta[i] - pp;              // ((I - P^+ P) Abar)_i
        double pb[6];
        for (int q = 0; q < 6; ++q) pb[q] = -u[q] * A[i] + r[q] * pu + z[q] * qi;
        xb[i] = pb[1] + 2.0 * x[i] * pb[3] + y[i] * pb[4];
        yb[i] = pb[2] + x[i] * pb[4] + 2.0 * y[i] * pb[5];
    }
}

// Minimal-image offset of slot s from the node, in FP64 from positions of type P.
template <typename P>
__device__ __forceinline__ void offset64(const void *pos, int s, double xn, double yn,
                                         double &dx, double &dy)
{
    P px, py;
    load_pos((const P *)pos, s, px, py);
    dx = wrap1((double)px - xn);
    dy = wrap1((double)py - yn);
}

template <typename P, typename V, typename R, int SHAPE, bool POS>
__global__ void __launch_bounds__(64) k_bwd_fix(BwdArgs b)
{
    const P2MArgs &a = b.f;
    const int cnt = min(*a.defer_count, a.defer_cap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < cnt; it += gridDim.x * blockDim.x) {
        const long long node = a.defer_list[it];
        const int I = (int)(node % a.n), J = (int)(node / a.n);
        const int nc = a.n - 1;
        const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
        int *oslot = b.e_slot + node * b.K;
        R *ow = (R *)b.e_w + node * b.K;
        R *od = POS ? (R *)b.e_dpos + node * b.K * 2 : nullptr;
        double g[8];
        for (int c = 0; c < 8; ++c)
            g[c] = c < a.C ? (double)load_val<V, R>((const V *)b.grad_mesh + node * a.C + c) : 0.0;
        constexpr int UM = UMAX_SVD;
        int us[UM];
        double uw[UM], ub[UM], udx[UM], udy[UM];
        int nu = 0, vi[3], tri[3];
        unsigned vm[3] = {0u, 0u, 0u};
        const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
        int stars[3][KMAX];
        int ns[3] = {0, 0, 0};
        int st = locate(a.B, qn, a.R0, tri, stars[0], ns[0]);
        if (SHAPE == PFEM_SHAPE_QUADRATIC)
            for (int e = 0; e < 3 && st == 0; ++e)
                if (ns[e] == 0) {
                    const int c = star_of(a.B, tri[e], a.R0, stars[e]);
                    if (c < 0) st = c;
                    else ns[e] = c;
                }
        if (st == 0) {
            bool over = false;
            auto add = [&](int s) -> int {
                for (int i = 0; i < nu; ++i)
                    if (us[i] == s) return i;
                if (nu == UM || nu == b.K) { over = true; return 0; }
                us[nu] = s;
                uw[nu] = udx[nu] = udy[nu] = 0.0;
                return nu++;
            };
            for (int e = 0; e < 3; ++e) vi[e] = add(tri[e]);
            if (SHAPE == PFEM_SHAPE_QUADRATIC)
                for (int e = 0; e < 3; ++e) {
                    unsigned m = 1u << vi[e];
                    for (int i = 0; i < ns[e]; ++i) m |= 1u << add(stars[e][i]);
                    vm[e] = m;
                }
            if (over) st = -PFEM_ERR_CAPACITY;
        }
        if (st == 0) {
            // offsets from the node in FP64 (FP32 positions promoted, as the forward fix pass does)
            NodePos<P, R> np;
            np.init(Iu, Ju, nc);
            double ox[UM], oy[UM];
            for (int i = 0; i < nu; ++i) {
                R dx, dy;
                np.off(a.pos, us[i], dx, dy);
                ox[i] = (double)dx;
                oy[i] = (double)dy;
                R v[8];
                load_vals<V, R>((const V *)a.vals, a.perm, us[i], a.C, v);
                double t = 0.0;
                for (int c = 0; c < 8; ++c)
                    if (c < a.C) t = fma(g[c], (double)v[c], t);
                ub[i] = t;
            }
            double d[3][2];
            for (int e = 0; e < 3; ++e) { d[e][0] = ox[vi[e]]; d[e][1] = oy[vi[e]]; }
            const double Na = d[1][0] * d[2][1] - d[1][1] * d[2][0];
            const double Nb = d[2][0] * d[0][1] - d[2][1] * d[0][0];
            const double Nc = d[0][0] * d[1][1] - d[0][1] * d[1][0];
            const double A2 = Na + Nb + Nc;
            const double lam[3] = {Na / A2, Nb / A2, Nc / A2};
            double lbar[3];
            for (int e = 0; e < 3; ++e) {
                uw[vi[e]] += lam[e];
                lbar[e] = ub[vi[e]];
            }
            if (SHAPE == PFEM_SHAPE_QUADRATIC)
                for (int e = 0; e < 3; ++e) {
                    const int f = e == 2 ? 0 : e + 1;
                    const unsigned mask = vm[e] | vm[f];
                    const double mx = 0.5 * (d[e][0] + d[f][0]), my = 0.5 * (d[e][1] + d[f][1]);
                    const double ex = d[e][0] - d[f][0], ey = d[e][1] - d[f][1];
                    const double sl = sqrt(ex * ex + ey * ey), inv = 1.0 / sl;
                    const double tx = ex * inv, ty = ey * inv;
                    double pt[UM][6], x[UM], y[UM], be[UM], A[UM], xb[UM], yb[UM];
                    int ids[UM];
                    int k = 0;
                    for (unsigned m = mask; m; m &= m - 1) {
                        const int i = __ffs(m) - 1;
                        x[k] = (ox[i] - mx) * inv;
                        y[k] = (oy[i] - my) * inv;
                        pt[k][0] = 1.0; pt[k][1] = x[k]; pt[k][2] = y[k];
                        pt[k][3] = x[k] * x[k]; pt[k][4] = x[k] * y[k]; pt[k][5] = y[k] * y[k];
                        be[k] = ub[i];
                        ids[k++] = i;
                    }
                    const double bv[6] = {0.0, 0.0, 0.0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
                    const double ce = 2.0 * lam[e] * lam[f];
                    double bb[6], Be;
                    edge_adjoint_svd(k, pt, x, y, be, bv, ce, A, xb, yb, bb, Be);
                    for (int j = 0; j < k; ++j) uw[ids[j]] = fma(ce, A[j], uw[ids[j]]);
                    lbar[e] += 2.0 * lam[f] * Be;
                    lbar[f] += 2.0 * lam[e] * Be;
                    if (POS) {
                        // members: x = (o - m) / s; frame: m = (d_e + d_f) / 2, s = |d_e - d_f|
                        double mbx = 0.0, mby = 0.0, sb = 0.0;
                        for (int j = 0; j < k; ++j) {
                            udx[ids[j]] += xb[j] * inv;
                            udy[ids[j]] += yb[j] * inv;
                            mbx -= xb[j] * inv;
                            mby -= yb[j] * inv;
                            sb -= (xb[j] * x[j] + yb[j] * y[j]) * inv;
                        }
                        // b = -(1/2) [tx^2, tx ty, ty^2] with t = (d_e - d_f) / s
                        const double tbx = -tx * bb[3] - 0.5 * ty * bb[4];
                        const double tby = -0.5 * tx * bb[4] - ty * bb[5];
                        const double tt = tbx * tx + tby * ty;
                        const double ebx = (tbx - tt * tx) * inv + sb * tx;
                        const double eby = (tby - tt * ty) * inv + sb * ty;
                        udx[vi[e]] += 0.5 * mbx + ebx;
                        udy[vi[e]] += 0.5 * mby + eby;
                        udx[vi[f]] += 0.5 * mbx - ebx;
                        udy[vi[f]] += 0.5 * mby - eby;
                    }
                }
            if (POS) {
                // lambda_k = N_k / A2 with N_a = d_b x d_c, N_b = d_c x d_a, N_c = d_a x d_b
                const double Lam = lbar[0] * lam[0] + lbar[1] * lam[1] + lbar[2] * lam[2];
                const double n0 = (lbar[0] - Lam) / A2, n1 = (lbar[1] - Lam) / A2,
                             n2 = (lbar[2] - Lam) / A2;
                double gx[3] = {0.0, 0.0, 0.0}, gy[3] = {0.0, 0.0, 0.0};
                gx[1] += n0 * d[2][1];  gy[1] -= n0 * d[2][0];
                gx[2] -= n0 * d[1][1];  gy[2] += n0 * d[1][0];
                gx[2] += n1 * d[0][1];  gy[2] -= n1 * d[0][0];
                gx[0] -= n1 * d[2][1];  gy[0] += n1 * d[2][0];
                gx[0] += n2 * d[1][1];  gy[0] -= n2 * d[1][0];
                gx[1] -= n2 * d[0][1];  gy[1] += n2 * d[0][0];
                for (int e = 0; e < 3; ++e) {
                    udx[vi[e]] += gx[e];
                    udy[vi[e]] += gy[e];
                }
            }
        }
        if (st != 0) {
            if (st == -PFEM_FAR) st = -PFEM_ERR_CAPACITY;
            record_error(a.status, -st, node);
            nu = 0;
        }
        for (int k = 0; k < b.K; ++k) {
            const bool v = k < nu;
            oslot[k] = v ? us[k] : -1;
            ow[k] = v ? (R)uw[k] : R(0);
            if (POS) {
                od[2 * k] = v ? (R)udx[k] : R(0);
                od[2 * k + 1] = v ? (R)udy[k] : R(0);
            }
        }
    }
}

// ---------------------------------------------------------------- transposed gather

__global__ void k_tr_count(long long E, const int *__restrict__ slot, int *__restrict__ count,
                           int *__restrict__ rank)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = slot[e];
        rank[e] = s >= 0 ? atomicAdd(count + s, 1) : -1;
    }
}

__global__ void k_tr_scatter(long long E, const int *__restrict__ slot, const int *__restrict__ rank,
                             const int *__restrict__ start, int *__restrict__ order)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = slot[e];
        if (s >= 0) order[__ldg(start + s) + rank[e]] = (int)e;
    }
}

__global__ void k_tr_sort(long long N, const int *__restrict__ start, int *order)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int a = start[s], b = start[s + 1];
        for (int i = a + 1; i < b; ++i) {
            const int v = order[i];
            int j = i - 1;
            while (j >= a && order[j] > v) {
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = v;
        }
    }
}

// grad_vals[particle] = sum_e w_e gbar_node(e); grad_pos[particle] = sum_e dpos_e
template <typename V, typename R, typename W>
__global__ void k_tr_gather(long long N, int K, int C, const int *__restrict__ start,
                            const int *__restrict__ order, const W *__restrict__ ew,
                            const R *__restrict__ edpos, const V *__restrict__ grad_mesh,
                            const int *__restrict__ perm, V *__restrict__ grad_vals,
                            V *__restrict__ grad_pos)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        R gv[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) gv[c] = R(0);
        R gx = R(0), gy = R(0);
        const int a = __ldg(start + s), b = __ldg(start + s + 1);
        for (int i = a; i < b; ++i) {
            const int e = __ldg(order + i);
            const long long node = e / K;
            const R w = (R)__ldg(ew + e);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < C) gv[c] = fma(w, load_val<V, R>(grad_mesh + node * C + c), gv[c]);
            if (edpos) {
                gx += __ldg(edpos + 2LL * e);
                gy += __ldg(edpos + 2LL * e + 1);
            }
        }
        const long long o = perm ? (long long)__ldg(perm + s) : s;
        if (grad_vals)
            for (int c = 0; c < C; ++c) store_val<V, R>(grad_vals + o * C + c, gv[c]);
        if (grad_pos && edpos) {
            store_val<V, R>(grad_pos + 2 * o, gx);
            store_val<V, R>(grad_pos + 2 * o + 1, gy);
        }
    }
}

static unsigned grid1(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > num_sms() * 64LL) b = num_sms() * 64LL;
    return (unsigned)b;
}

BwdLayout bwd_layout(int n, long long N, int Kw)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    BwdLayout L;
    L.K = KBWD;
    const int K = Kw > KBWD ? Kw : KBWD;
    const long long E = (long long)n * n * K;
    size_t off = 256;
    L.e_slot = off;  off = al(off + 4 * (size_t)E);
    L.e_w = off;     off = al(off + 8 * (size_t)E);
    L.e_dpos = off;  off = al(off + 16 * (size_t)E);
    L.count = off;   off = al(off + 4 * (size_t)(N + 1));
    L.start = off;   off = al(off + 4 * (size_t)(N + 1));
    L.rank = off;    off = al(off + 4 * (size_t)E);
    L.order = off;   off = al(off + 4 * (size_t)E);
    L.scan = off;    off = al(off + 4 * scan_scratch_ints(N + 1));
    NodeRecs r;
    L.rec = off;     off = al(off + node_recs_layout(nullptr, (long long)n * n, &r));
    L.tab = off;     off = al(off + star_tab_bytes(N));
    L.queue = off;   off = al(off + 8 * (size_t)n * n);
    L.total = off;
    return L;
}

// Phase 2 over entries (slot, w, dpos) laid out [n*n, K].
template <typename V, typename R, typename W>
static cudaError_t transposed_gather(int n, long long N, int K, int C, const int *e_slot,
                                     const W *e_w, const R *e_dpos, const void *grad_mesh,
                                     const int *perm, void *grad_vals, void *grad_pos,
                                     const BwdLayout &L, char *ws, cudaStream_t s)
{
    const long long E = (long long)n * n * K;
    int *count = (int *)(ws + L.count);
    int *start = (int *)(ws + L.start);
    int *rank = (int *)(ws + L.rank);
    int *order = (int *)(ws + L.order);
    cudaError_t e = cudaMemsetAsync(count, 0, 4 * (size_t)(N + 1), s);
    if (e != cudaSuccess) return e;
    k_tr_count<<<grid1(E, 256), 256, 0, s>>>(E, e_slot, count, rank);
    count_launch();
    e = scan_exclusive(count, start, N + 1, (int *)(ws + L.scan), s);
    if (e != cudaSuccess) return e;
    k_tr_scatter<<<grid1(E, 256), 256, 0, s>>>(E, e_slot, rank, start, order);
    k_tr_sort<<<grid1(N, 128), 128, 0, s>>>(N, start, order);
    k_tr_gather<V, R, W><<<grid1(N, 128), 128, 0, s>>>(N, K, C, start, order, e_w, e_dpos,
                                                       (const V *)grad_mesh, perm, (V *)grad_vals,
                                                       (V *)grad_pos);
    count_launch(3);
    return cudaGetLastError();
}

template <typename P, typename V, typename R, typename S, int SHAPE>
static cudaError_t bwd_t(const GeoArgs &g, const int *perm, int C, const void *vals,
                         const void *grad_mesh, void *grad_vals, void *grad_pos, bool checkpoint,
                         const int *w_idx, const void *w, int Kw, const BwdLayout &L, char *ws,
                         cudaStream_t s)
{
    const int K = L.K;
    BwdArgs b;
    b.f.n = g.n;
    b.f.B.q = (const uint2 *)g.q_sorted;
    b.f.B.start = g.cell_start;
    b.f.B.nb = g.nb;
    b.f.B.rmax = g.rmax;
    b.f.B.dmax = g.dmax;
    b.f.B.kcap = g.kcap;
    b.f.B.walk_cap = g.walk_cap;
    b.f.ucap = g.ucap;
    b.f.R0 = g.R0;
    b.f.pos = g.pos_sorted;
    b.f.perm = perm;
    b.f.vals = vals;
    b.f.C = C;
    b.f.out = nullptr;
    b.f.w_idx = nullptr;
    b.f.w = nullptr;
    b.f.K = 0;
    b.f.status = (DevStatus *)ws;
    b.grad_mesh = grad_mesh;
    b.K = K;
    b.e_slot = (int *)(ws + L.e_slot);
    b.e_w = ws + L.e_w;
    b.e_dpos = ws + L.e_dpos;
    const dim3 grid((g.n + 15) / 16, (g.n + 7) / 8);
    // per-node adjoint entries: the geometry and solve kernels for FP32 quadratic solves, else
    // the single fused kernel
    NodeRecs recs;
    node_recs_layout(ws + L.rec, (long long)g.n * g.n, &recs);
    // the star table's queue counter sits in the status block, after the status word
    const StarTab tab = star_tab_layout(ws + L.tab, g.N, (int *)(ws + 64));
    const bool split = SHAPE == PFEM_SHAPE_QUADRATIC && sizeof(S) == sizeof(float);
    // the fix-pass queue: its counter in the status block, one entry per node
    b.f.defer_count = (int *)(ws + 68);
    b.f.defer_list = (long long *)(ws + L.queue);
    b.f.defer_cap = (int)std::min((long long)g.n * g.n, (long long)0x7fffffff);
    auto node_pass = [&](bool pos) {
        cudaMemsetAsync(b.f.defer_count, 0, sizeof(int), s);
        if (split) {
            launch_star_table(b.f.B, g.R0, g.rmax_far, tab, b.f.status, s);
            k_p2m_geom<P, V, R><<<grid, 128, 0, s>>>(b.f, tab, recs);
            const unsigned blocks = (unsigned)((recs.nodes + 127) / 128);
            if (pos) k_bwd_solve<P, V, R, S, true><<<blocks, 128, 0, s>>>(b, recs);
            else k_bwd_solve<P, V, R, S, false><<<blocks, 128, 0, s>>>(b, recs);
            count_launch(2);
        } else {
            if (pos) k_bwd_node<P, V, R, S, SHAPE, true><<<grid, 128, 0, s>>>(b);
            else k_bwd_node<P, V, R, S, SHAPE, false><<<grid, 128, 0, s>>>(b);
            count_launch();
        }
        // the queued nodes: widest search radius, FP64 SVD adjoint
        BwdArgs bf = b;
        bf.f.B.rmax = std::max(g.rmax, g.rmax_far);
        if (pos) k_bwd_fix<P, V, R, SHAPE, true><<<num_sms() * 2, 64, 0, s>>>(bf);
        else k_bwd_fix<P, V, R, SHAPE, false><<<num_sms() * 2, 64, 0, s>>>(bf);
        count_launch();
    };
    if (checkpoint) {
        // value gradient straight from the stored weights
        cudaError_t e = transposed_gather<V, R, R>(g.n, g.N, Kw, C, w_idx, (const R *)w,
                                                   (const R *)nullptr, grad_mesh, perm, grad_vals,
                                                   nullptr, L, ws, s);
        if (e != cudaSuccess || !grad_pos) return e;
        node_pass(true);
        return transposed_gather<V, R, R>(g.n, g.N, K, C, b.e_slot, (const R *)b.e_w,
                                          (const R *)b.e_dpos, grad_mesh, perm, nullptr, grad_pos,
                                          L, ws, s);
    }
    if (!grad_pos) b.e_dpos = nullptr;
    node_pass(grad_pos != nullptr);
    return transposed_gather<V, R, R>(g.n, g.N, K, C, b.e_slot, (const R *)b.e_w,
                                      grad_pos ? (const R *)b.e_dpos : nullptr, grad_mesh, perm,
                                      grad_vals, grad_pos, L, ws, s);
}

cudaError_t launch_p2m_backward(const GeoArgs &g, const int *perm, int C, const void *vals,
                                pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                bool checkpoint, const int *w_idx, const void *w, int Kw,
                                const void *grad_mesh, void *grad_vals, void *grad_pos,
                                const BwdLayout &L, void *ws, cudaStream_t s)
{
    char *W = (char *)ws;
    const bool q = shape == PFEM_SHAPE_QUADRATIC;
    if (val_t == PFEM_F64) {
        if (q) return bwd_t<double, double, double, double, 1>(g, perm, C, vals, grad_mesh, grad_vals, grad_pos, checkpoint, w_idx, w, Kw, L, W, s);
        return bwd_t<double, double, double, double, 0>(g, perm, C, vals, grad_mesh, grad_vals, grad_pos, checkpoint, w_idx, w, Kw, L, W, s);
    }
    if (!q) return bwd_t<float, float, float, float, 0>(g, perm, C, vals, grad_mesh, grad_vals, grad_pos, checkpoint, w_idx, w, Kw, L, W, s);
    if (solve == PFEM_SOLVE_F64)
        return bwd_t<float, float, float, double, 1>(g, perm, C, vals, grad_mesh, grad_vals, grad_pos, checkpoint, w_idx, w, Kw, L, W, s);
    return bwd_t<float, float, float, float, 1>(g, perm, C, vals, grad_mesh, grad_vals, grad_pos, checkpoint, w_idx, w, Kw, L, W, s);
}

}  // namespace pfem
