// p2m.cuh -- per-node particle-to-mesh projection (Sec. 2.2 eq. p2m) with linear FE or
// quadratically consistent shape functions (App. B eq. phiquad), one thread per mesh node.
//
// For node r_i in the particle Delaunay triangle T = (a, b, c) with barycentrics lambda, the
// only nonzero linear shape functions are lambda_a, lambda_b, lambda_c, and eq. (phiquad)
// sums A_{mu nu sigma} phi_nu phi_sigma over ordered pairs of distinct, adjacent nu, sigma --
// the three edges of T, each twice.  So
//     w_{i mu} = lambda_mu [mu in T] + sum_{e=(nu,sigma) in T} 2 lambda_nu lambda_sigma A_{mu e},
// and alpha_i = sum_mu w_{i mu} alpha_mu for every field component in one pass.
#pragma once

#include "geom.cuh"
#include "moments.cuh"
#include "startab.cuh"

namespace pfem {

struct P2MArgs {
    int n;                      // mesh nodes per side (image row/column included)
    Bins B;
    int R0;                     // first search radius in bins
    const void *pos;            // [N,2] positions in slot order
    const int *perm;            // slot -> original index, or nullptr (values in slot order)
    const void *vals;           // [N,C]
    int C;
    void *out;                  // [n,n,C] mesh values (apply mode)
    int *w_idx;                 // [n*n, K] (weights mode)
    void *w;                    // [n*n, K]
    int K;
    DevStatus *status;
    // Queue of nodes whose moment system the fast solve could not factor (rank deficient, or
    // too ill-conditioned for its precision), recomputed by k_p2m_fix; capacity 0 = no queue.
    int *defer_count = nullptr;
    long long *defer_list = nullptr;
    int defer_cap = 0;
    // Index of this problem's first node in a batch (0 for one problem): queue entries and
    // error details are node indices of the whole batch.
    long long noff = 0;
    int ucap = PFEM_UMAX;       // distinct particles of one node in the fast pass
};

// node_quadratic's code for "queue this node for the FP64 SVD pass" (not a public status), and
// the marker of a node that was queued.
constexpr int PFEM_DEFER = 64;
constexpr int PFEM_DEFERRED = 1;

// A node whose moment system the fast solve could not factor, or whose search ran out of its
// region (-PFEM_FAR), is queued for the fix pass (FP64, SVD solve, widest search radius) and
// returns PFEM_DEFERRED; with no queue (the fix pass itself, or a workspace without room) it
// becomes PFEM_ERR_DEGENERATE or PFEM_ERR_CAPACITY.
__device__ __forceinline__ int defer_or_error(const P2MArgs &a, int st, long long node)
{
    if (st != -PFEM_DEFER && st != -PFEM_FAR) return st;
    if (a.defer_cap <= 0) return st == -PFEM_FAR ? -PFEM_ERR_CAPACITY : -PFEM_ERR_DEGENERATE;
    const int i = atomicAdd(a.defer_count, 1);
    if (i >= a.defer_cap) return -PFEM_ERR_CAPACITY;
    a.defer_list[i] = node;
    return PFEM_DEFERRED;
}

// Minimum-norm least-squares solution of P A = b (App. A: the SVD with rank detection), for the
// 6 x k matrix P whose columns are the stencil's monomial vectors; pt holds P^T (k rows of 6,
// k <= SVD_ROWS) and is overwritten.  jacobi_svd gives P^T V = W with orthogonal columns
// w_j = sigma_j u_j (left in pt), V orthogonal and sig2[j] = sigma_j^2; then P = V W^T and
// A = sum_j (v_j . b / sigma_j^2) w_j over the singular values above max(k, 6) eps sigma_max
// (smaller ones are rank deficiency).
//
// Steps: a Householder QR P^T = Q [R; 0] (Golub & Van Loan, 5.2), which keeps the singular
// values; one-sided (Hestenes) Jacobi on the 6 x 6 factor R -- plane rotations of pairs of its
// columns until all are mutually orthogonal, accumulated in V, so that R V = W6 -- with R, V and
// the rotations in registers; then W = Q [W6; 0].  The sweeps, the long part, so run on 6 rows
// instead of k.
constexpr int SVD_ROWS = 32;

// Householder QR of pt (k x 6): R (6 x 6; rows past min(k, 6) zero) and the reflections, v_j
// kept in pt[j..k-1][j] with vv[j] = v_j . v_j (0: no reflection).
static __device__ __forceinline__ void householder_qr(int k, double (*pt)[6], double R[6][6],
                                                      double vv[6])
{
    const int m = k < 6 ? k : 6;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) R[i][j] = 0.0;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        vv[j] = 0.0;
        if (j >= m) continue;
        double nx = 0.0;
        for (int i = j; i < k; ++i) nx = fma(pt[i][j], pt[i][j], nx);
        const double x0 = pt[j][j];
        const double alpha = x0 >= 0.0 ? -sqrt(nx) : sqrt(nx);
        if (nx > 0.0) {
            pt[j][j] = x0 - alpha;
            vv[j] = 2.0 * (nx + fabs(x0) * sqrt(nx));     // v.v = 2 (|x|^2 - alpha x0)
#pragma unroll
            for (int c = j + 1; c < 6; ++c) {
                double d = 0.0;
                for (int i = j; i < k; ++i) d = fma(pt[i][j], pt[i][c], d);
                const double f = 2.0 * d / vv[j];
                for (int i = j; i < k; ++i) pt[i][c] = fma(-f, pt[i][j], pt[i][c]);
            }
        }
        R[j][j] = nx > 0.0 ? alpha : x0;
#pragma unroll
        for (int c = j + 1; c < 6; ++c) R[j][c] = pt[j][c];
    }
}

// out[0..k) = Q [y; 0] = H_0 H_1 ... H_5 [y; 0] with the reflections of householder_qr.
static __device__ __forceinline__ void apply_q(int k, const double (*pt)[6], const double vv[6],
                                               const double y[6], double *out)
{
    for (int i = 0; i < k; ++i) out[i] = i < 6 ? y[i] : 0.0;
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        if (vv[j] == 0.0) continue;
        double d = 0.0;
        for (int i = j; i < k; ++i) d = fma(pt[i][j], out[i], d);
        const double f = 2.0 * d / vv[j];
        for (int i = j; i < k; ++i) out[i] = fma(-f, pt[i][j], out[i]);
    }
}

// One-sided (Hestenes) Jacobi on R (6 x 6): plane rotations of pairs of its columns until all
// are mutually orthogonal, accumulated in V, so that R V = W6 (left in R), sig2[j] = |w6_j|^2.
//  - Each sweep takes the 15 column pairs in the round-robin order of 5 rounds of 3 disjoint
//    pairs, so that three rotations are independent.
//  - A rotation's tangent comes from FP32 arithmetic: any exact rotation keeps the singular
//    values, and its angle only sets how fast the off-diagonal products fall.  c = 1/sqrt(1+t^2)
//    and s = c t are formed in FP64 from that t, so the rotation is orthogonal to FP64
//    precision.  (FP64 divides and square roots are long instruction sequences on the narrow
//    FP64 pipe.)
//  - Columns whose squared norm is below 1e-31 of ||R||_F^2 are left alone: the rank detection
//    drops them (its threshold is above (6 eps)^2 sigma_max^2 >= 1.7e-30 ||R||_F^2 / 6), and their
//    rounding noise would otherwise keep a sweep from converging.
static __device__ __forceinline__ void jacobi6(double R[6][6], double V[6][6], double sig2[6])
{
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    double f2 = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 6; ++j) f2 = fma(R[i][j], R[i][j], f2);
    const double tiny2 = 1e-31 * f2;
    constexpr int RR[5][3][2] = {{{0, 1}, {2, 3}, {4, 5}}, {{0, 2}, {1, 4}, {3, 5}},
                                 {{0, 3}, {1, 5}, {2, 4}}, {{0, 4}, {1, 3}, {2, 5}},
                                 {{0, 5}, {1, 2}, {3, 4}}};
    for (int sweep = 0; sweep < 40; ++sweep) {
        bool rotated = false;
#pragma unroll
        for (int r = 0; r < 5; ++r) {
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const int p = RR[r][h][0], q = RR[r][h][1];
                double al = 0.0, be = 0.0, ga = 0.0;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    al = fma(R[i][p], R[i][p], al);
                    be = fma(R[i][q], R[i][q], be);
                    ga = fma(R[i][p], R[i][q], ga);
                }
                if (!(ga * ga > 1e-30 * al * be) || al < tiny2 || be < tiny2) continue;
                // tangent of the rotation angle: zeta = (be - al) / (2 ga), in FP32 while the
                // operands are well inside its range (near-coincident particles can make the
                // scaled monomials huge), else in FP64
                double t;
                const double dba = be - al;
                // binary exponents from the bit patterns (integer pipes): |dba| < 2^96 and
                // 2^-95 <= |ga| < 2^96
                const int ed = (__double2hiint(dba) >> 20) & 0x7ff, eg = (__double2hiint(ga) >> 20) & 0x7ff;
                if (ed < 1023 + 96 && eg > 1023 - 96 && eg < 1023 + 96) {
                    const float gf = f32_trunc(ga), df = f32_trunc(dba);
                    const float zf = df / (2.f * gf);
                    const float tf = copysignf(1.f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.f)));
                    if (!(tf != 0.f)) continue; // |zeta| beyond 1e19: the angle is below FP64's
                    t = f64_of(tf);
                } else {
                    const double zeta = dba / (2.0 * ga);
                    t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                    if (!(t != 0.0)) continue;
                }
                rotated = true;
                const double c = rsqrt(fma(t, t, 1.0)), s = c * t;
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const double x = R[i][p], y = R[i][q];
                    R[i][p] = fma(c, x, -s * y);
                    R[i][q] = fma(s, x, c * y);
                    const double u = V[i][p], w = V[i][q];
                    V[i][p] = fma(c, u, -s * w);
                    V[i][q] = fma(s, u, c * w);
                }
            }
        }
        if (!rotated) break;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        double s2 = 0.0;
#pragma unroll
        for (int i = 0; i < 6; ++i) s2 = fma(R[i][j], R[i][j], s2);
        sig2[j] = s2;
    }
}

// The SVD P^T V = W of the k x 6 matrix in pt (overwritten with W): householder_qr, jacobi6 on
// R, then W = Q [W6; 0].
static __device__ __forceinline__ void jacobi_svd(int k, double (*pt)[6], double V[6][6],
                                                  double sig2[6])
{
    double R[6][6], vv[6];
    householder_qr(k, pt, R, vv);
    jacobi6(R, V, sig2);
    double W[SVD_ROWS][6];
    for (int i = 0; i < k; ++i)
#pragma unroll
        for (int c = 0; c < 6; ++c) W[i][c] = i < 6 ? R[i][c] : 0.0;
#pragma unroll
    for (int j = 5; j >= 0; --j) {
        if (vv[j] == 0.0) continue;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            double d = 0.0;
            for (int i = j; i < k; ++i) d = fma(pt[i][j], W[i][c], d);
            const double f = 2.0 * d / vv[j];
            for (int i = j; i < k; ++i) W[i][c] = fma(-f, pt[i][j], W[i][c]);
        }
    }
    for (int i = 0; i < k; ++i)
#pragma unroll
        for (int c = 0; c < 6; ++c) pt[i][c] = W[i][c];
}

// Squared singular values kept by the rank detection: above (max(k, 6) eps)^2 sigma_max^2.
__device__ __forceinline__ double svd_threshold2(int k, const double sig2[6])
{
    double smax2 = 0.0;
    for (int j = 0; j < 6; ++j) smax2 = fmax(smax2, sig2[j]);
    const double tol = (double)(k > 6 ? k : 6) * 2.220446049250313e-16;
    return tol * tol * smax2;
}

static __device__ __noinline__ void minnorm_lsq(int k, double (*pt)[6], const double b[6],
                                                double *A)
{
    // A = sum_j (v_j . b / sigma_j^2) w_j = Q [sum_j (v_j . b / sigma_j^2) w6_j; 0]
    double R[6][6], vv[6], V[6][6], sig2[6];
    householder_qr(k, pt, R, vv);
    jacobi6(R, V, sig2);
    const double thr2 = svd_threshold2(k, sig2);
    double z[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        if (!(sig2[j] > thr2)) continue;
        double d = 0.0;
#pragma unroll
        for (int r = 0; r < 6; ++r) d = fma(V[r][j], b[r], d);
        const double cj = d / sig2[j];
#pragma unroll
        for (int i = 0; i < 6; ++i) z[i] = fma(cj, R[i][j], z[i]);
    }
    apply_q(k, pt, vv, z, A);
}

// Node position and minimal-image offsets in the compute precision R.
template <typename P, typename R> struct NodePos;

template <> struct NodePos<double, double> {
    double x, y;
    __device__ __forceinline__ void init(int Iu, int Ju, int nc)
    {
        x = (double)Iu / (double)nc;
        y = (double)Ju / (double)nc;
    }
    __device__ __forceinline__ void off(const void *pos, int s, double &dx, double &dy) const
    {
        double px, py;
        load_pos((const double *)pos, s, px, py);
        dx = wrap1(px - x);
        dy = wrap1(py - y);
    }
};

// FP32 offsets: the node coordinate I/nc is carried as hi + lo, so that an offset is accurate
// to FP32 relative precision (px - hi is exact for nearby values, and wraps exactly).
template <> struct NodePos<float, float> {
    float xh, xl, yh, yl;
    __device__ __forceinline__ void init(int Iu, int Ju, int nc)
    {
        const float f = (float)nc;
        xh = (float)Iu / f;
        xl = fmaf(-xh, f, (float)Iu) / f;
        yh = (float)Ju / f;
        yl = fmaf(-yh, f, (float)Ju) / f;
    }
    __device__ __forceinline__ void off(const void *pos, int s, float &dx, float &dy) const
    {
        float px, py;
        load_pos((const float *)pos, s, px, py);
        dx = wrap1(px - xh) - xl;
        dy = wrap1(py - yh) - yl;
    }
};

template <typename V, typename R>
__device__ __forceinline__ void load_vals(const V *vals, const int *perm, int s, int C, R out[8])
{
    const long long idx = perm ? (long long)__ldg(perm + s) : (long long)s;
    const V *p = vals + idx * C;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < C) out[c] = load_val<V, R>(p + c);
}

template <>
__device__ __forceinline__ void load_vals<float, float>(const float *vals, const int *perm, int s,
                                                        int C, float out[8])
{
    const long long idx = perm ? (long long)__ldg(perm + s) : (long long)s;
    if (C == 4 && (reinterpret_cast<uintptr_t>(vals) & 15) == 0) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(vals) + idx);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
        return;
    }
    const float *p = vals + idx * C;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < C) out[c] = __ldg(p + c);
}

template <typename V, typename R>
__device__ __forceinline__ void store_vals(V *out, long long node, int C, const R acc[8])
{
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < C) store_val<V, R>(out + node * C + c, acc[c]);
}

template <>
__device__ __forceinline__ void store_vals<float, float>(float *out, long long node, int C,
                                                        const float acc[8])
{
    if (C == 4 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        reinterpret_cast<float4 *>(out)[node] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        return;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (c < C) out[node * C + c] = acc[c];
}

// A star as a plain array of slots (the stars a thread searched itself).
struct ArrStar {
    const int *p;
    int n;
    __device__ __forceinline__ int operator[](int i) const { return p[i]; }
};

// Quadratic weights of one node over its distinct particles U = T + stars of T's vertices:
// offsets are loaded once per particle, each edge's stencil is a bit mask over U, and
// w_u = lambda_u [u in T] + sum_e 2 lambda_nu lambda_sg A_{u e} accumulates per particle.
// Calls emit(slot, w) once per particle of U.  Returns 0, -PFEM_DEFER (a moment matrix the
// Cholesky solve cannot factor, or more than UMAX distinct particles: queue the node for the
// SVD pass) or, in the SVD pass, -PFEM_ERR_CAPACITY (more than UMAX_SVD distinct particles).
constexpr int UMAX = PFEM_UMAX; // fast pass: jittered lattices have at most about 20
constexpr int UMAX_SVD = 32;   // SVD pass (the stencil masks are 32-bit)
static_assert(UMAX_SVD <= SVD_ROWS, "stencils of the SVD pass fit jacobi_svd's rows");

// SVD = true (the FP64 pass over queued nodes): each edge's coefficients are the minimum-norm
// least-squares solution by SVD instead of the Cholesky solve of the moment system.
// The node's distinct particles U = T + stars of T's vertices (slots us[0..nu)), the stencil
// of the edge (tri[e], tri[e+1]) as the bit mask vm[e] | vm[e+1] over U, vi[e] the index of
// tri[e] in U, and uw initialised to the linear weights lambda.  Returns 0, or -1 when U has
// more than UM particles.
template <int UM, typename R, typename SA>
__device__ __forceinline__ int node_u_build(const int tri[3], const SA *st, const R lam[3],
                                            int *us, R *uw, int &nu, unsigned vm[3], int vi[3],
                                            int cap = UM)
{
    nu = 0;
    bool over = false;
    auto add = [&](int s) -> int {
        for (int i = 0; i < nu; ++i)
            if (us[i] == s) return i;
        if (nu == cap) { over = true; return 0; }
        us[nu] = s;
        uw[nu] = R(0);
        return nu++;
    };
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        vi[e] = add(tri[e]);
        uw[vi[e]] += lam[e];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        unsigned m = 1u << vi[e];
        for (int i = 0; i < st[e].n; ++i) m |= 1u << add(st[e][i]);
        vm[e] = m;
    }
    return over ? -1 : 0;
}

// node_u_build without the weights: the particle set and the stencil masks only.
template <int UM, typename SA>
__device__ __forceinline__ int node_u_sets(const int tri[3], const SA *st, int *us, int &nu,
                                           unsigned vm[3], int vi[3], int cap = UM)
{
    nu = 0;
    bool over = false;
    auto add = [&](int s) -> int {
        for (int i = 0; i < nu; ++i)
            if (us[i] == s) return i;
        if (nu == cap) { over = true; return 0; }
        us[nu] = s;
        return nu++;
    };
#pragma unroll
    for (int e = 0; e < 3; ++e) vi[e] = add(tri[e]);
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        unsigned m = 1u << vi[e];
        for (int i = 0; i < st[e].n; ++i) m |= 1u << add(st[e][i]);
        vm[e] = m;
    }
    return over ? -1 : 0;
}

// The three edge systems of a node over its particle set: uw[u] += 2 lambda_nu lambda_sg A_{u e}.
// Returns 0, or -PFEM_DEFER when a moment matrix is below the fast-solve tolerance.
template <typename P, typename R, typename S, int REFINE, bool SVD, int UM>
__device__ __forceinline__ int node_u_solve(const P2MArgs &a, const NodePos<P, R> &np,
                                            const int *us, R *uw, const unsigned vm[3],
                                            const int vi[3], const R lam[3])
{
    // Offsets are re-read from the positions, which neighbouring nodes share in L1, instead of
    // being copied into thread-private memory.
    auto offset = [&](int i, S &x, S &y) {
        R dx, dy;
        np.off(a.pos, us[i], dx, dy);
        x = S(dx);
        y = S(dy);
    };
    // The three edges in a loop that is not unrolled: one copy of the edge code keeps the
    // kernels' instruction footprint and register spills down (fused kernel with the refined
    // solve: 1.047 -> 1.010 ms at 1025^2 nodes / 2048^2 particles; spills 164 -> 40 bytes).
#ifndef PFEM_EDGE_UNROLL
#define PFEM_EDGE_UNROLL 1
#endif
    constexpr int edge_unroll = PFEM_EDGE_UNROLL;
#pragma unroll edge_unroll
    for (int e = 0; e < 3; ++e) {
        const int f = e == 2 ? 0 : e + 1;
        const unsigned mask = vm[e] | vm[f];
        S rnx, rny, rsx, rsy;
        offset(vi[e], rnx, rny);
        offset(vi[f], rsx, rsy);
        const S mx = (rnx + rsx) * S(0.5), my = (rny + rsy) * S(0.5);
        const S ex = rnx - rsx, ey = rny - rsy;
        const S inv = S(1) / sqrt(ex * ex + ey * ey);
        if constexpr (SVD) {
            double pt[UM][6];
            int ids[UM];
            int k = 0;
            for (unsigned m = mask; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                S ox, oy;
                offset(i, ox, oy);
                const double x = (double)((ox - mx) * inv), y = (double)((oy - my) * inv);
                pt[k][0] = 1.0; pt[k][1] = x; pt[k][2] = y;
                pt[k][3] = x * x; pt[k][4] = x * y; pt[k][5] = y * y;
                ids[k++] = i;
            }
            const double tx = (double)(ex * inv), ty = (double)(ey * inv);
            const double b[6] = {0.0, 0.0, 0.0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
            double A[UM];
            minnorm_lsq(k, pt, b, A);
            const double coef = 2.0 * (double)lam[e] * (double)lam[f];
            for (int j = 0; j < k; ++j) uw[ids[j]] += (R)(coef * A[j]);
            continue;
        }
        Moment<S> M;
        M.zero();
        for (unsigned m = mask; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            S ox, oy;
            offset(i, ox, oy);
            M.add((ox - mx) * inv, (oy - my) * inv);
        }
        if (!M.factor(FastTol<S>::v)) return -PFEM_DEFER;
        const S tx = ex * inv, ty = ey * inv;
        const S b[6] = {S(0), S(0), S(0), S(-0.5) * tx * tx, S(-0.5) * tx * ty, S(-0.5) * ty * ty};
        S y[6];
        M.solve(b, y);
        if constexpr (REFINE == REFINE_FF) {
            // r = b - sum_mu p_mu (p_mu . y) in float-float, with the monomials of the FP32
            // offsets formed exactly (the same system the FP64 residual refines)
            FF r[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) r[k] = {(float)b[k], 0.f};
            for (unsigned m = mask; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                S ox, oy;
                offset(i, ox, oy);
                const float X = (float)((ox - mx) * inv), Y = (float)((oy - my) * inv);
                const FF p[6] = {{1.f, 0.f}, {X, 0.f}, {Y, 0.f}, ff_two_prod(X, X),
                                 ff_two_prod(X, Y), ff_two_prod(Y, Y)};
                FF t = {(float)y[0], 0.f};
#pragma unroll
                for (int k = 1; k < 6; ++k) t = ff_add(t, ff_mul(p[k], (float)y[k]));
#pragma unroll
                for (int k = 0; k < 6; ++k) r[k] = ff_add(r[k], ff_neg(ff_mul(p[k], t)));
            }
            S rs[6], dy[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) rs[k] = (S)(r[k].h + r[k].l);
            M.solve(rs, dy);
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] += dy[k];
        }
        if constexpr (REFINE == REFINE_F64) {
            // r = b - sum_mu p_mu (p_mu . y) in FP64: t = p . y by nested products, and the
            // monomial terms of r as X (X t), Y (X t), Y (Y t)
            double r[6], yd[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                r[k] = f64_of(b[k]);
                yd[k] = f64_of(y[k]);
            }
            for (unsigned m = mask; m; m &= m - 1) {
                const int i = __ffs(m) - 1;
                S ox, oy;
                offset(i, ox, oy);
                const double X = f64_of((ox - mx) * inv), Y = f64_of((oy - my) * inv);
                const double t = fma(X, fma(X, yd[3], fma(Y, yd[4], yd[1])),
                                     fma(Y, fma(Y, yd[5], yd[2]), yd[0]));
                const double xt = X * t, yt = Y * t;
                r[0] -= t;
                r[1] -= xt;
                r[2] -= yt;
                r[3] = fma(-X, xt, r[3]);
                r[4] = fma(-Y, xt, r[4]);
                r[5] = fma(-Y, yt, r[5]);
            }
            S rs[6], dy[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) rs[k] = f32_trunc(r[k]);
            M.solve(rs, dy);
#pragma unroll
            for (int k = 0; k < 6; ++k) y[k] += dy[k];
        }
        const R coef = R(2) * lam[e] * lam[f];
        for (unsigned m = mask; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            S ox, oy;
            offset(i, ox, oy);
            const S x = (ox - mx) * inv, yv = (oy - my) * inv;
            const S A = y[0] + x * y[1] + yv * y[2] + x * x * y[3] + x * yv * y[4] + yv * yv * y[5];
            uw[i] = fma(coef, R(A), uw[i]);
        }
    }
    return 0;
}

template <typename P, typename R, typename S, int REFINE, bool SVD = false, typename SA,
          typename Emit>
__device__ __forceinline__ int node_quadratic(const P2MArgs &a, const NodePos<P, R> &np,
                                              const int tri[3], const SA *st, const R lam[3],
                                              Emit &&emit)
{
    constexpr int UM = SVD ? UMAX_SVD : UMAX;
    int us[UM];
    R uw[UM];
    int nu;
    unsigned vm[3];
    int vi[3];
    if (node_u_build<UM>(tri, st, lam, us, uw, nu, vm, vi, SVD ? UM : min(a.ucap, UM)) != 0)
        return SVD ? -PFEM_ERR_CAPACITY : -PFEM_DEFER;
    const int r = node_u_solve<P, R, S, REFINE, SVD, UM>(a, np, us, uw, vm, vi, lam);
    if (r != 0) return r;
    for (int i = 0; i < nu; ++i) emit(us[i], uw[i]);
    return 0;
}

// Barycentric coordinates of the node (the origin of np's offsets) in triangle tri.
template <typename P, typename R>
__device__ __forceinline__ void barycentric(const P2MArgs &a, const NodePos<P, R> &np,
                                            const int tri[3], R lam[3])
{
    R d[3][2];
#pragma unroll
    for (int e = 0; e < 3; ++e) np.off(a.pos, tri[e], d[e][0], d[e][1]);
    const R area2 = (d[1][0] - d[0][0]) * (d[2][1] - d[0][1]) - (d[1][1] - d[0][1]) * (d[2][0] - d[0][0]);
    lam[0] = (d[1][0] * d[2][1] - d[1][1] * d[2][0]) / area2;
    lam[1] = (d[2][0] * d[0][1] - d[2][1] * d[0][0]) / area2;
    lam[2] = (d[0][0] * d[1][1] - d[0][1] * d[1][0]) / area2;
}

template <typename V> __device__ __forceinline__ V nan_of();
template <> __device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double nan_of<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// One mesh node.  WEIGHTS = false: write alpha_i for all C components; true: write the
// node's distinct (slot, weight) pairs.
template <typename P, typename V, typename R, typename S, int REFINE, int SHAPE, bool WEIGHTS,
          bool SVD = false>
__device__ __forceinline__ void p2m_node(const P2MArgs &a, int I, int J)
{
    const int nc = a.n - 1;
    const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
    const long long node = (long long)J * a.n + I;
    const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
    int tri[3];
    int stars[3][KMAX];
    int ns[3] = {0, 0, 0};
    int st = locate(a.B, qn, a.R0, tri, stars[0], ns[0]);
    if (SHAPE == PFEM_SHAPE_QUADRATIC && st == 0) {
        for (int e = 0; e < 3 && st == 0; ++e)
            if (ns[e] == 0) {
                const int c = star_of(a.B, tri[e], a.R0, stars[e]);
                if (c < 0) st = c;
                else ns[e] = c;
            }
    }
    NodePos<P, R> np;
    np.init(Iu, Ju, nc);
    R lam[3] = {R(0), R(0), R(0)};
    if (st == 0) barycentric(a, np, tri, lam);

    if (!WEIGHTS) {
        R acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = R(0);
        auto emit = [&](int s, R wgt) {
            R v[8];
            load_vals<V, R>((const V *)a.vals, a.perm, s, a.C, v);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < a.C) acc[c] = fma(wgt, v[c], acc[c]);
        };
        if (st == 0) {
            if (SHAPE == PFEM_SHAPE_QUADRATIC) {
                const ArrStar sa[3] = {{stars[0], ns[0]}, {stars[1], ns[1]}, {stars[2], ns[2]}};
                st = node_quadratic<P, R, S, REFINE, SVD>(a, np, tri, sa, lam, emit);
            } else {
                for (int e = 0; e < 3; ++e) emit(tri[e], lam[e]);
            }
        }
        st = defer_or_error(a, st, a.noff + node);
        if (st != 0) {
            if (st < 0) record_error(a.status, -st, a.noff + node);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
        }
        store_vals<V, R>((V *)a.out, node, a.C, acc);
    } else {
        int idx[PFEM_KW_MAX];
        R wl[PFEM_KW_MAX];
        int cnt = 0;
        bool over = false;
        auto emit = [&](int s, R wgt) {
            for (int i = 0; i < cnt; ++i)
                if (idx[i] == s) { wl[i] += wgt; return; }
            if (cnt < a.K) { idx[cnt] = s; wl[cnt] = wgt; ++cnt; }
            else over = true;
        };
        if (st == 0) {
            if (SHAPE == PFEM_SHAPE_QUADRATIC) {
                const ArrStar sa[3] = {{stars[0], ns[0]}, {stars[1], ns[1]}, {stars[2], ns[2]}};
                st = node_quadratic<P, R, S, REFINE, SVD>(a, np, tri, sa, lam, emit);
            } else {
                for (int e = 0; e < 3; ++e) emit(tri[e], lam[e]);
            }
            if (over && st == 0) st = -PFEM_ERR_CAPACITY;
        }
        st = defer_or_error(a, st, a.noff + node);
        if (st != 0) {
            if (st < 0) record_error(a.status, -st, a.noff + node);
            cnt = 0;
        }
        int *oi = a.w_idx + node * a.K;
        R *ow = (R *)a.w + node * a.K;
        for (int k = 0; k < a.K; ++k) {
            oi[k] = k < cnt ? idx[k] : -1;
            ow[k] = k < cnt ? wl[k] : R(0);
        }
    }
}

// Resident blocks per SM the compiler must allow (it caps registers at 65536 / (128 x 12) = 42):
// the per-node work is latency-bound, and measured on GB300 (sweep 1..16) twelve 128-thread
// blocks per SM were fastest despite the extra register spills.
#ifndef PFEM_P2M_MIN_BLOCKS
#define PFEM_P2M_MIN_BLOCKS 12
#endif

template <typename P, typename V, typename R, typename S, int REFINE, int SHAPE, bool WEIGHTS>
__global__ void __launch_bounds__(128, PFEM_P2M_MIN_BLOCKS) k_p2m(P2MArgs a)
{
    const int I = blockIdx.x * 16 + (threadIdx.x & 15);
    const int J = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (I >= a.n || J >= a.n) return;
    p2m_node<P, V, R, S, REFINE, SHAPE, WEIGHTS>(a, I, J);
}

// The queued nodes again, overwriting the fast pass's placeholder output: the geometry searched
// per thread with the widest search radius (the launcher passes it in a.B.rmax), and with
// quadratic shape functions every edge solved in FP64 by the SVD.  A node that fails here
// reports its error.
template <typename P, typename V, typename R, int SHAPE, bool WEIGHTS>
__global__ void __launch_bounds__(128) k_p2m_fix(P2MArgs a)
{
    const int cnt = min(*a.defer_count, a.defer_cap);
    P2MArgs f = a;
    f.defer_cap = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const long long node = a.defer_list[i];
        p2m_node<P, V, R, double, REFINE_NONE, SHAPE, WEIGHTS, true>(
            f, (int)(node % a.n), (int)(node / a.n));
    }
}

// ---------------------------------------------------------------- two-kernel P2M
// The table path as two kernels, each with its own register budget: k_p2m_geom locates the node
// and builds its particle set from the star table (memory latency bound), k_p2m_solve solves the
// three edge systems and applies the weights.  They hand over a per-node record, one array per
// field so that both kernels access it coalesced.  The float-float solve and the adjoint take
// this form; the other forward solves run both halves in k_p2m_tab.
struct NodeRecs {
    int *meta;          // [nodes] nu | vi0 << 5 | vi1 << 10 | vi2 << 15, or -1: no record
    unsigned *mask;     // [3][nodes] vm[e]
    double *lam;        // [3][nodes] barycentric coordinates (exact in both precisions)
    int *us;            // [UMAX][nodes] slots of the particle set
    long long *loc;     // [nodes] Iu | Ju << 21 | nc << 42 (batches of problems), or null
    long long nodes;
};

// Lays the record arrays for `nodes` nodes out from `base` (256-byte aligned arrays; base may be
// null to size them); returns the bytes they take.
inline size_t node_recs_layout(char *base, long long nodes, NodeRecs *r, bool with_loc = false)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_meta = 0;
    const size_t o_mask = al(o_meta + sizeof(int) * (size_t)nodes);
    const size_t o_lam = al(o_mask + 3 * sizeof(unsigned) * (size_t)nodes);
    const size_t o_us = al(o_lam + 3 * sizeof(double) * (size_t)nodes);
    const size_t o_loc = al(o_us + UMAX * sizeof(int) * (size_t)nodes);
    const size_t total = with_loc ? al(o_loc + sizeof(long long) * (size_t)nodes) : o_loc;
    if (base) {
        r->meta = (int *)(base + o_meta);
        r->mask = (unsigned *)(base + o_mask);
        r->lam = (double *)(base + o_lam);
        r->us = (int *)(base + o_us);
        r->loc = with_loc ? (long long *)(base + o_loc) : nullptr;
    }
    r->nodes = nodes;
    return total;
}

// Resident 128-thread blocks per SM of the geometry kernel: its node search waits on memory,
// and more warps in flight hide it (8, 10, 12, 16 blocks measured 0.291, 0.275, 0.268, 0.266 ms
// at 1025^2 nodes / 2048^2 particles); 12 keeps the register spills to a few dozen bytes.
#ifndef PFEM_GEOM_MIN_BLOCKS
#define PFEM_GEOM_MIN_BLOCKS 12
#endif
// Node (I, J) of the mesh of a.n nodes per side: locate it and build its particle set from the
// star table, and write its record at index `rec` (node J * a.n + I of a single problem; the
// problem's offset plus that in a batch, which also records the node's coordinates).
template <typename P, typename V, typename R>
__device__ __forceinline__ void geom_node(const P2MArgs &a, const StarTab &t, const NodeRecs &r,
                                          int I, int J, long long rec)
{
    const int nc = a.n - 1;
    const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
    const long long node = (long long)J * a.n + I;
    const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
    int tri[3];
    int st = locate_tab(a.B, t, qn, a.R0, tri);
    TabStar sa[3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
        if (st == 0) {
            sa[e] = tab_star(t, tri[e]);
            if (sa[e].n < 0) st = sa[e].n == -1 ? -PFEM_FAR : sa[e].n;
        }
    int meta = -1;
    if (st == 0) {
        NodePos<P, R> np;
        np.init(Iu, Ju, nc);
        R lam[3];
        barycentric(a, np, tri, lam);
        int us[UMAX];
        int nu;
        unsigned vm[3];
        int vi[3];
        if (node_u_sets<UMAX>(tri, sa, us, nu, vm, vi, min(a.ucap, UMAX)) != 0) {
            st = a.defer_cap > 0 ? -PFEM_DEFER : -PFEM_ERR_CAPACITY;
        } else {
            // entries up to the warp's largest set, -1 past this node's, so that the warp's
            // stores to each entry array cover contiguous runs of it
            const int nw = __reduce_max_sync(__activemask(), nu);
            for (int i = 0; i < nw; ++i) r.us[i * r.nodes + rec] = i < nu ? us[i] : -1;
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                r.mask[e * r.nodes + rec] = vm[e];
                r.lam[e * r.nodes + rec] = (double)lam[e];
            }
            meta = nu | vi[0] << 5 | vi[1] << 10 | vi[2] << 15;
        }
    }
    r.meta[rec] = meta;
    if (r.loc) r.loc[rec] = (long long)Iu | (long long)Ju << 21 | (long long)nc << 42;
    if (st != 0) {
        st = defer_or_error(a, st, rec);
        if (st < 0) record_error(a.status, -st, rec);
        if (a.out) {                    // the adjoint uses this kernel without a mesh output
            R acc[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
            store_vals<V, R>((V *)a.out, node, a.C, acc);
        }
    }
}

template <typename P, typename V, typename R>
__global__ void __launch_bounds__(128, PFEM_GEOM_MIN_BLOCKS) k_p2m_geom(P2MArgs a, StarTab t,
                                                                        NodeRecs r)
{
    const int I = blockIdx.x * 16 + (threadIdx.x & 15);
    const int J = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (I >= a.n || J >= a.n) return;
    geom_node<P, V, R>(a, t, r, I, J, (long long)J * a.n + I);
}

// The fix pass of the table path: the queued nodes located with the star table (complete after
// the retry kernels; the launcher passes the widest search radius for the nearest particle) and
// every edge solved in FP64 by the SVD, as k_p2m_fix does with stars searched per thread.  With
// CHOL (runs whose fast pass solved in FP32) a node first takes the FP64 Cholesky solve of the
// FP64 fast path, pivot tolerance included: a system too ill-conditioned for the FP32 solve is
// usually well within FP64's, and only the nodes below that tolerance (rank deficient, or
// conditioned beyond it) take the SVD.
template <typename P, typename V, typename R, bool CHOL>
__global__ void __launch_bounds__(128) k_p2m_fix_tab(P2MArgs a, StarTab t)
{
    const int cnt = min(*a.defer_count, a.defer_cap);
    P2MArgs f = a;
    f.defer_cap = 0;
    const int nc = a.n - 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const long long node = a.defer_list[i];
        const int I = (int)(node % a.n), J = (int)(node / a.n);
        const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
        const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
        int tri[3];
        int st = locate_tab(f.B, t, qn, f.R0, tri);
        if (st == -PFEM_FAR) st = -PFEM_ERR_CAPACITY;
        TabStar sa[3];
#pragma unroll
        for (int e = 0; e < 3; ++e)
            if (st == 0) {
                sa[e] = tab_star(t, tri[e]);
                if (sa[e].n < 0) st = sa[e].n == -1 ? -PFEM_ERR_CAPACITY : sa[e].n;
            }
        NodePos<P, R> np;
        np.init(Iu, Ju, nc);
        R acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = R(0);
        if (st == 0) {
            R lam[3];
            barycentric(f, np, tri, lam);
            auto emit = [&](int sl, R wgt) {
                R v[8];
                load_vals<V, R>((const V *)f.vals, f.perm, sl, f.C, v);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c < f.C) acc[c] = fma(wgt, v[c], acc[c]);
            };
            st = CHOL ? node_quadratic<P, R, double, REFINE_NONE, false>(f, np, tri, sa, lam, emit)
                      : -PFEM_DEFER;
            if (st == -PFEM_DEFER)      // nothing was emitted
                st = node_quadratic<P, R, double, REFINE_NONE, true>(f, np, tri, sa, lam, emit);
        }
        if (st != 0) {
            record_error(f.status, -st, node);
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
        }
        store_vals<V, R>((V *)f.out, node, f.C, acc);
    }
}

// Resident 128-thread blocks per SM of the solve kernel (the two-kernel form: the float-float
// refinement): 8 (64 registers) for the FP32 moment system (sweep 8, 10, 12: 8), and 8 as well
// for the refined solves with the edge loop rolled (float-float: 6 -> 8 blocks 0.553 -> 0.536
// ms at 1025^2 nodes / 2048^2 particles).  A refined solve needs many warps in flight to keep
// the FP64 pipe busy: one to three persistent blocks per SM measured 1.1 to 2.4 times slower.
#ifndef PFEM_SOLVE_MIN_BLOCKS
#define PFEM_SOLVE_MIN_BLOCKS 8
#endif
#ifndef PFEM_SOLVE_REF_MIN_BLOCKS
#define PFEM_SOLVE_REF_MIN_BLOCKS 8
#endif
template <typename S, int REFINE> constexpr int solve_min_blocks()
{
    return sizeof(S) == 8 ? 4 : REFINE != REFINE_NONE ? PFEM_SOLVE_REF_MIN_BLOCKS : PFEM_SOLVE_MIN_BLOCKS;
}

template <typename P, typename V, typename R, typename S, int REFINE>
__global__ void __launch_bounds__(128, solve_min_blocks<S, REFINE>()) k_p2m_solve(P2MArgs a, NodeRecs r)
{
    const long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (node >= r.nodes) return;
    const int meta = r.meta[node];
    if (meta < 0) return;
    const int nu = meta & 31;
    const int vi[3] = {(meta >> 5) & 31, (meta >> 10) & 31, (meta >> 15) & 31};
    int us[UMAX];
    R uw[UMAX];
    for (int i = 0; i < nu; ++i) {
        us[i] = r.us[i * r.nodes + node];
        uw[i] = R(0);
    }
    unsigned vm[3];
    R lam[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        vm[e] = r.mask[e * r.nodes + node];
        lam[e] = (R)r.lam[e * r.nodes + node];
        uw[vi[e]] += lam[e];
    }
    NodePos<P, R> np;
    if (r.loc) {                        // batch: the node's own mesh, output at its record index
        const long long l = r.loc[node];
        np.init((int)(l & 0x1fffff), (int)((l >> 21) & 0x1fffff), (int)(l >> 42));
    } else {
        const int nc = a.n - 1;
        const int I = (int)(node % a.n), J = (int)(node / a.n);
        np.init(I == nc ? 0 : I, J == nc ? 0 : J, nc);
    }
    int st = node_u_solve<P, R, S, REFINE, false, UMAX>(a, np, us, uw, vm, vi, lam);
    R acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = R(0);
    if (st == 0) {
        for (int i = 0; i < nu; ++i) {
            R v[8];
            load_vals<V, R>((const V *)a.vals, a.perm, us[i], a.C, v);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < a.C) acc[c] = fma(uw[i], v[c], acc[c]);
        }
    } else {
        st = defer_or_error(a, st, node);
        if (st < 0) record_error(a.status, -st, node);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
    }
    store_vals<V, R>((V *)a.out, node, a.C, acc);
}

// The table path's fast pass in one kernel: each thread locates its node with the star table,
// builds its particle set and solves its three edge systems, without a node record in between.
// The refined solve is bound by the FP64 pipe, which leaves the other pipes and the memory
// system to the location work of the other warps.
// Resident blocks per SM of k_p2m_tab with the refined solve: 8 (64 registers; with the edge
// loop rolled 6, 7, 8 measured 1.051, 1.011, 1.000 ms at 1025^2 nodes / 2048^2 particles).
#ifndef PFEM_TAB_REF_MIN_BLOCKS
#define PFEM_TAB_REF_MIN_BLOCKS 8
#endif
template <typename S, int REFINE> constexpr int tab_min_blocks()
{
    return sizeof(S) == 8 || REFINE == REFINE_NONE ? solve_min_blocks<S, REFINE>() : PFEM_TAB_REF_MIN_BLOCKS;
}

// Node (I, J) of the problem of a (mesh output a.out; queue entries and error details at node
// a.noff + J * a.n + I of the batch).
template <typename P, typename V, typename R, typename S, int REFINE>
__device__ __forceinline__ void tab_node(const P2MArgs &a, const StarTab &t, int I, int J)
{
    const int nc = a.n - 1;
    const int Iu = I == nc ? 0 : I, Ju = J == nc ? 0 : J;
    const long long node = (long long)J * a.n + I;
    const uint2 qn = make_uint2(node_fx(Iu, nc), node_fx(Ju, nc));
    int tri[3];
    int st = locate_tab(a.B, t, qn, a.R0, tri);
    TabStar sa[3];
#pragma unroll
    for (int e = 0; e < 3; ++e)
        if (st == 0) {
            sa[e] = tab_star(t, tri[e]);
            if (sa[e].n < 0) st = sa[e].n == -1 ? -PFEM_FAR : sa[e].n;
        }
    R acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = R(0);
    if (st == 0) {
        NodePos<P, R> np;
        np.init(Iu, Ju, nc);
        R lam[3];
        barycentric(a, np, tri, lam);
        int us[UMAX];
        int nu;
        unsigned vm[3];
        int vi[3];
        if (node_u_sets<UMAX>(tri, sa, us, nu, vm, vi, min(a.ucap, UMAX)) != 0) {
            st = a.defer_cap > 0 ? -PFEM_DEFER : -PFEM_ERR_CAPACITY;
        } else {
            R uw[UMAX];
            for (int i = 0; i < nu; ++i) uw[i] = R(0);
#pragma unroll
            for (int e = 0; e < 3; ++e) uw[vi[e]] += lam[e];
            st = node_u_solve<P, R, S, REFINE, false, UMAX>(a, np, us, uw, vm, vi, lam);
            if (st == 0)
                for (int i = 0; i < nu; ++i) {
                    R v[8];
                    load_vals<V, R>((const V *)a.vals, a.perm, us[i], a.C, v);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c < a.C) acc[c] = fma(uw[i], v[c], acc[c]);
                }
        }
    }
    if (st != 0) {
        st = defer_or_error(a, st, a.noff + node);
        if (st < 0) record_error(a.status, -st, a.noff + node);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
    }
    store_vals<V, R>((V *)a.out, node, a.C, acc);
}

template <typename P, typename V, typename R, typename S, int REFINE>
__global__ void __launch_bounds__(128, tab_min_blocks<S, REFINE>()) k_p2m_tab(P2MArgs a, StarTab t)
{
    const int I = blockIdx.x * 16 + (threadIdx.x & 15);
    const int J = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (I >= a.n || J >= a.n) return;
    tab_node<P, V, R, S, REFINE>(a, t, I, J);
}

}  // namespace pfem
