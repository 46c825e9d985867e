// m2p.cu -- mesh-to-particle interpolation (Sec. 2.2 eq. m2p) with linear FE shape functions
// on the fixed structured mesh: one thread per particle, in the caller's particle order.
//
// The particle's cell (i, j) comes from its fixed-point coordinates (the same rule that bins
// the particles); local coordinates s = x/H - i, t = y/H - j select the triangle of the cell
// split along (i,j)->(i+1,j+1):
//   s >= t: weights (1-s, s-t, t) on nodes (i,j), (i+1,j), (i+1,j+1)
//   s <  t: weights (1-t, s, t-s) on nodes (i,j), (i+1,j+1), (i,j+1)
// Because the image row and column are stored, i+1 and j+1 never wrap.  The kernel is a
// bandwidth-bound gather: positions and outputs stream once; the mesh is read through L2.
#include <cmath>

#include "internal.h"

namespace pfem {

template <typename R> __device__ __forceinline__ R local_coord(R x, int i, int nc)
{
    const R xw = x - floor(x);                          // exact
    R s = fma(xw, (R)nc, (R)(-i));
    if (s > (R)(0.5 * nc)) s -= (R)nc;                  // fixed point rounded up to 2^32 -> cell 0
    return s;
}

template <typename P, typename V, typename R, int CT>
__global__ void __launch_bounds__(256) k_m2p(int n, long long N, const P *__restrict__ pos,
                                             int Crt, const V *__restrict__ mesh,
                                             V *__restrict__ vals)
{
    const int C = CT > 0 ? CT : Crt;
    const int nc = n - 1;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x) {
        P px, py;
        load_pos(pos, m, px, py);
        const int i = bin_of(fx_of(px), nc), j = bin_of(fx_of(py), nc);
        const P s = local_coord<P>(px, i, nc), t = local_coord<P>(py, j, nc);
        const long long n00 = (long long)j * n + i;
        long long nb_, nc_;
        R w0, w1, w2;
        if (s >= t) { nb_ = n00 + 1; nc_ = n00 + n + 1; w0 = R(P(1) - s); w1 = R(s - t); w2 = R(t); }
        else        { nb_ = n00 + n + 1; nc_ = n00 + n; w0 = R(P(1) - t); w1 = R(s); w2 = R(t - s); }
        if constexpr (CT == 4 && sizeof(V) == 4 && sizeof(R) == 4) {
            const float4 a = __ldg(reinterpret_cast<const float4 *>(mesh) + n00);
            const float4 b = __ldg(reinterpret_cast<const float4 *>(mesh) + nb_);
            const float4 c = __ldg(reinterpret_cast<const float4 *>(mesh) + nc_);
            float4 o;
            o.x = fmaf(w0, a.x, fmaf(w1, b.x, w2 * c.x));
            o.y = fmaf(w0, a.y, fmaf(w1, b.y, w2 * c.y));
            o.z = fmaf(w0, a.z, fmaf(w1, b.z, w2 * c.z));
            o.w = fmaf(w0, a.w, fmaf(w1, b.w, w2 * c.w));
            __stcs(reinterpret_cast<float4 *>(vals) + m, o);
        } else {
            for (int c = 0; c < C; ++c) {
                const R v = w0 * load_val<V, R>(mesh + n00 * C + c) +
                            w1 * load_val<V, R>(mesh + nb_ * C + c) +
                            w2 * load_val<V, R>(mesh + nc_ * C + c);
                store_val<V, R>(vals + m * C + c, v);
            }
        }
    }
}

template <typename P, typename V, typename R>
static cudaError_t m2p_t(int n, long long N, const void *pos, int C, const void *mesh, void *vals,
                         cudaStream_t s)
{
    long long blocks = (N + 255) / 256;
    if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
    if (blocks < 1) blocks = 1;
    const bool aligned = ((reinterpret_cast<uintptr_t>(mesh) | reinterpret_cast<uintptr_t>(vals)) & 15) == 0;
    if (C == 4 && aligned)
        k_m2p<P, V, R, 4><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const P *)pos, C,
                                                          (const V *)mesh, (V *)vals);
    else
        k_m2p<P, V, R, 0><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const P *)pos, C,
                                                          (const V *)mesh, (V *)vals);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2p(int n, long long N, const void *pos, pfem_dtype pos_t, int C,
                       const void *mesh, void *vals, pfem_dtype val_t, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    if (val_t == PFEM_F64) {
        if (pos_t == PFEM_F64) return m2p_t<double, double, double>(n, N, pos, C, mesh, vals, s);
        return m2p_t<float, double, double>(n, N, pos, C, mesh, vals, s);
    }
    if (val_t == PFEM_F32) {
        if (pos_t == PFEM_F64) return m2p_t<double, float, float>(n, N, pos, C, mesh, vals, s);
        return m2p_t<float, float, float>(n, N, pos, C, mesh, vals, s);
    }
    if (pos_t == PFEM_F64) return m2p_t<double, __nv_bfloat16, float>(n, N, pos, C, mesh, vals, s);
    return m2p_t<float, __nv_bfloat16, float>(n, N, pos, C, mesh, vals, s);
}

// ---------------------------------------------------------------- adjoint of M2P

// grad_mesh[node] = sum over particles whose triangle uses this stored node of w * gbar.
// One thread per stored node; particles of the (up to four) cells around it are visited in
// bin order, so the sum order is fixed (no atomics).  Stored image entries receive only the
// reads that the forward made from them.
template <typename P, typename V, typename R>
__global__ void __launch_bounds__(128) k_m2p_bwd_mesh(int n, int nb, const P *__restrict__ pos,
                                                      const int *__restrict__ cell_start,
                                                      const int *__restrict__ perm, int C,
                                                      const V *__restrict__ gv,
                                                      V *__restrict__ gm)
{
    const int I = blockIdx.x * 16 + (threadIdx.x & 15);
    const int J = blockIdx.y * 8 + (threadIdx.x >> 4);
    if (I >= n || J >= n) return;
    const int nc = n - 1;
    const long long node = (long long)J * n + I;
    R acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = R(0);
    for (int cj = J - 1; cj <= J; ++cj) {
        if (cj < 0 || cj >= nc) continue;
        const long long ylo = bin_lo(cj, nc), yhi = bin_lo(cj + 1, nc);
        const int by0 = bin_of((uint32_t)ylo, nb), by1 = bin_of((uint32_t)(yhi - 1), nb);
        for (int ci = I - 1; ci <= I; ++ci) {
            if (ci < 0 || ci >= nc) continue;
            const long long xlo = bin_lo(ci, nc), xhi = bin_lo(ci + 1, nc);
            const int bx0 = bin_of((uint32_t)xlo, nb), bx1 = bin_of((uint32_t)(xhi - 1), nb);
            for (int by = by0; by <= by1; ++by) {
                const int s0 = __ldg(cell_start + (long long)by * nb + bx0);
                const int s1 = __ldg(cell_start + (long long)by * nb + bx1 + 1);
                for (int s = s0; s < s1; ++s) {
                    const int m = __ldg(perm + s);
                    P px, py;
                    load_pos(pos, m, px, py);
                    const int i = bin_of(fx_of(px), nc), j = bin_of(fx_of(py), nc);
                    if (i != ci || j != cj) continue;
                    const P ss = local_coord<P>(px, i, nc), tt = local_coord<P>(py, j, nc);
                    const long long n00 = (long long)j * n + i;
                    R w = R(0);
                    if (ss >= tt) {
                        if (node == n00) w = R(P(1) - ss);
                        else if (node == n00 + 1) w = R(ss - tt);
                        else if (node == n00 + n + 1) w = R(tt);
                    } else {
                        if (node == n00) w = R(P(1) - tt);
                        else if (node == n00 + n + 1) w = R(ss);
                        else if (node == n00 + n) w = R(tt - ss);
                    }
                    if (w == R(0)) continue;
                    for (int c = 0; c < C; ++c)
                        acc[c] = fma(w, load_val<V, R>(gv + (long long)m * C + c), acc[c]);
                }
            }
        }
    }
    for (int c = 0; c < C; ++c) store_val<V, R>(gm + node * C + c, acc[c]);
}

// grad_pos[m] = sum_c gbar_c * grad f_c(r_m), f the linear FE interpolant of the mesh field.
template <typename P, typename V, typename R>
__global__ void __launch_bounds__(256) k_m2p_bwd_pos(int n, long long N, const P *__restrict__ pos,
                                                     int C, const V *__restrict__ mesh,
                                                     const V *__restrict__ gv, V *__restrict__ gp)
{
    const int nc = n - 1;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x) {
        P px, py;
        load_pos(pos, m, px, py);
        const int i = bin_of(fx_of(px), nc), j = bin_of(fx_of(py), nc);
        const P s = local_coord<P>(px, i, nc), t = local_coord<P>(py, j, nc);
        const long long n00 = (long long)j * n + i, n10 = n00 + 1, n11 = n00 + n + 1, n01 = n00 + n;
        R gx = R(0), gy = R(0);
        for (int c = 0; c < C; ++c) {
            const R g = load_val<V, R>(gv + m * C + c);
            const R f00 = load_val<V, R>(mesh + n00 * C + c), f10 = load_val<V, R>(mesh + n10 * C + c);
            const R f11 = load_val<V, R>(mesh + n11 * C + c), f01 = load_val<V, R>(mesh + n01 * C + c);
            R ds, dt;
            if (s >= t) { ds = f10 - f00; dt = f11 - f10; }
            else        { ds = f11 - f01; dt = f01 - f00; }
            gx = fma(g, ds, gx);
            gy = fma(g, dt, gy);
        }
        store_val<V, R>(gp + 2 * m, gx * (R)nc);
        store_val<V, R>(gp + 2 * m + 1, gy * (R)nc);
    }
}

template <typename P, typename V, typename R>
static cudaError_t m2p_bwd_t(int n, int nb, long long N, const void *pos, const int *cell_start,
                             const int *perm, int C, const void *mesh, const void *gv, void *gm,
                             void *gp, cudaStream_t s)
{
    k_m2p_bwd_mesh<P, V, R><<<dim3((n + 15) / 16, (n + 7) / 8), 128, 0, s>>>(
        n, nb, (const P *)pos, cell_start, perm, C, (const V *)gv, (V *)gm);
    count_launch();
    if (gp && N > 0) {
        long long blocks = (N + 255) / 256;
        if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
        k_m2p_bwd_pos<P, V, R><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const P *)pos, C,
                                                               (const V *)mesh, (const V *)gv,
                                                               (V *)gp);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_m2p_backward(int n, int nb, long long N, const void *pos, pfem_dtype pos_t,
                                const int *cell_start, const int *perm, int C, const void *mesh,
                                const void *gv, pfem_dtype val_t, void *gm, void *gp,
                                cudaStream_t s)
{
    if (val_t == PFEM_F64) {
        if (pos_t == PFEM_F64) return m2p_bwd_t<double, double, double>(n, nb, N, pos, cell_start, perm, C, mesh, gv, gm, gp, s);
        return m2p_bwd_t<float, double, double>(n, nb, N, pos, cell_start, perm, C, mesh, gv, gm, gp, s);
    }
    if (pos_t == PFEM_F64) return m2p_bwd_t<double, float, float>(n, nb, N, pos, cell_start, perm, C, mesh, gv, gm, gp, s);
    return m2p_bwd_t<float, float, float>(n, nb, N, pos, cell_start, perm, C, mesh, gv, gm, gp, s);
}

// ---------------------------------------------------------------- M2P with mesh QCSF
// Quadratically consistent mesh shape functions (App. B on the fixed mesh; the paper's
// projFEM6/projFEMq interpolate mesh -> particles with them, Table 1, and compute their
// coefficients once, Sec. 3.1).  With every cell split along (i,j)->(i+1,j+1), node (I,J) has
// neighbours (I+-1,J), (I,J+-1), (I+1,J+1), (I-1,J-1); an edge's stencil is the closed
// neighbourhood of both endpoints (10 nodes) and its minimum-norm coefficients depend only
// on the edge's direction.  For each of the two triangles of a cell the host folds the three
// edges into one table: the distinct stencil nodes (offsets from the cell corner), the
// coefficient of each node in each edge, and which nodes are the triangle's vertices.  Then
//   w_k = lambda_k [k vertex] + sum_e 2 lambda_P(e) lambda_Q(e) A_{k,e}.
// Node values are read at the unique nodes (I mod (n-1), J mod (n-1)).

constexpr int MQ_NODES = 16;

struct MQTable {
    int count[2];
    signed char ox[2][MQ_NODES], oy[2][MQ_NODES];
    signed char vertex[2][MQ_NODES];      // 0..2 = lambda index, -1 = not a vertex
    float A32[2][MQ_NODES][3];
    double A64[2][MQ_NODES][3];
    signed char ep[2][3], eq[2][3];       // edge e joins vertices ep[e], eq[e]
};

// Minimum-norm coefficients of the mesh edge from (0,0) to (ex,ey) over its 10-node
// stencil, by the 6x6 normal equations (FP64 Cholesky).
static int mesh_edge_host(int ex, int ey, int S[16][2], double A[16])
{
    static const int NB[6][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, -1}};
    int k = 0;
    const int ends[2][2] = {{0, 0}, {ex, ey}};
    for (int e = 0; e < 2; ++e)
        for (int m = -1; m < 6; ++m) {
            const int x = ends[e][0] + (m < 0 ? 0 : NB[m][0]);
            const int y = ends[e][1] + (m < 0 ? 0 : NB[m][1]);
            bool dup = false;
            for (int i = 0; i < k; ++i) dup |= S[i][0] == x && S[i][1] == y;
            if (!dup) { S[k][0] = x; S[k][1] = y; ++k; }
        }
    const double s = std::sqrt((double)(ex * ex + ey * ey));
    double P[16][6], M[6][6] = {{0}};
    for (int i = 0; i < k; ++i) {
        const double x = (S[i][0] - 0.5 * ex) / s, y = (S[i][1] - 0.5 * ey) / s;
        const double p[6] = {1, x, y, x * x, x * y, y * y};
        for (int r = 0; r < 6; ++r) {
            P[i][r] = p[r];
            for (int c = 0; c < 6; ++c) M[r][c] += p[r] * p[c];
        }
    }
    const double tx = ex / s, ty = ey / s;
    double b[6] = {0, 0, 0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
    double L[6][6] = {{0}};
    for (int j = 0; j < 6; ++j) {
        double d = M[j][j];
        for (int q = 0; q < j; ++q) d -= L[j][q] * L[j][q];
        L[j][j] = std::sqrt(d);
        for (int i = j + 1; i < 6; ++i) {
            double t = M[i][j];
            for (int q = 0; q < j; ++q) t -= L[i][q] * L[j][q];
            L[i][j] = t / L[j][j];
        }
    }
    double z[6], y[6];
    for (int r = 0; r < 6; ++r) {
        double t = b[r];
        for (int q = 0; q < r; ++q) t -= L[r][q] * z[q];
        z[r] = t / L[r][r];
    }
    for (int r = 5; r >= 0; --r) {
        double t = z[r];
        for (int q = r + 1; q < 6; ++q) t -= L[q][r] * y[q];
        y[r] = t / L[r][r];
    }
    for (int i = 0; i < k; ++i) {
        double a = 0;
        for (int r = 0; r < 6; ++r) a += P[i][r] * y[r];
        A[i] = a;
    }
    return k;
}

static MQTable build_mq_table()
{
    MQTable T;
    int S[3][16][2];
    double A[3][16];
    int K[3];
    const int D[3][2] = {{1, 0}, {0, 1}, {1, 1}};
    for (int t = 0; t < 3; ++t) K[t] = mesh_edge_host(D[t][0], D[t][1], S[t], A[t]);
    // triangle 0 (s >= t): (0,0), (1,0), (1,1); triangle 1: (0,0), (1,1), (0,1)
    const int V[2][3][2] = {{{0, 0}, {1, 0}, {1, 1}}, {{0, 0}, {1, 1}, {0, 1}}};
    for (int tr = 0; tr < 2; ++tr) {
        int cnt = 0;
        for (int i = 0; i < MQ_NODES; ++i) {
            T.vertex[tr][i] = -1;
            for (int e = 0; e < 3; ++e) { T.A32[tr][i][e] = 0.f; T.A64[tr][i][e] = 0.0; }
        }
        auto slot = [&](int x, int y) {
            for (int i = 0; i < cnt; ++i)
                if (T.ox[tr][i] == x && T.oy[tr][i] == y) return i;
            T.ox[tr][cnt] = (signed char)x;
            T.oy[tr][cnt] = (signed char)y;
            return cnt++;
        };
        for (int v = 0; v < 3; ++v) T.vertex[tr][slot(V[tr][v][0], V[tr][v][1])] = (signed char)v;
        for (int e = 0; e < 3; ++e) {
            const int f = (e + 1) % 3;
            int dx = V[tr][f][0] - V[tr][e][0], dy = V[tr][f][1] - V[tr][e][1];
            int bx = V[tr][e][0], by = V[tr][e][1];
            if (dx < 0 || dy < 0) { dx = -dx; dy = -dy; bx = V[tr][f][0]; by = V[tr][f][1]; }
            const int type = (dx == 1 && dy == 0) ? 0 : (dx == 0 && dy == 1) ? 1 : 2;
            T.ep[tr][e] = (signed char)e;
            T.eq[tr][e] = (signed char)f;
            for (int k = 0; k < K[type]; ++k) {
                const int i = slot(bx + S[type][k][0], by + S[type][k][1]);
                T.A64[tr][i][e] = A[type][k];
                T.A32[tr][i][e] = (float)A[type][k];
            }
        }
        T.count[tr] = cnt;
    }
    return T;
}

// built once per process (thread-safe initialisation of a function-local static)
static const MQTable &mq_table()
{
    static const MQTable T = build_mq_table();
    return T;
}

template <typename P, typename V, typename R, int CT>
__global__ void __launch_bounds__(256) k_m2p_q(int n, long long N, const P *__restrict__ pos, int Crt,
                                               const V *__restrict__ mesh, V *__restrict__ vals,
                                               const MQTable T)
{
    const int C = CT > 0 ? CT : Crt;
    const int nc = n - 1;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x) {
        P px, py;
        load_pos(pos, m, px, py);
        const int i = bin_of(fx_of(px), nc), j = bin_of(fx_of(py), nc);
        const P s = local_coord<P>(px, i, nc), t = local_coord<P>(py, j, nc);
        const int tr = s >= t ? 0 : 1;
        R lam[3];
        if (tr == 0) { lam[0] = R(P(1) - s); lam[1] = R(s - t); lam[2] = R(t); }
        else         { lam[0] = R(P(1) - t); lam[1] = R(s); lam[2] = R(t - s); }
        R ce[3];
#pragma unroll
        for (int e = 0; e < 3; ++e) ce[e] = R(2) * lam[T.ep[tr][e]] * lam[T.eq[tr][e]];
        R acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = R(0);
        const int cnt = T.count[tr];
        for (int k = 0; k < cnt; ++k) {
            R w;
            if (sizeof(R) == 8)
                w = R(T.A64[tr][k][0]) * ce[0] + R(T.A64[tr][k][1]) * ce[1] + R(T.A64[tr][k][2]) * ce[2];
            else
                w = R(T.A32[tr][k][0]) * ce[0] + R(T.A32[tr][k][1]) * ce[1] + R(T.A32[tr][k][2]) * ce[2];
            const int vk = T.vertex[tr][k];
            if (vk >= 0) w += lam[vk];
            int I = i + T.ox[tr][k], J = j + T.oy[tr][k];
            I += I < 0 ? nc : 0;
            I -= I >= nc ? nc : 0;
            J += J < 0 ? nc : 0;
            J -= J >= nc ? nc : 0;
            const long long node = (long long)J * n + I;
            if constexpr (CT == 4 && sizeof(V) == 4 && sizeof(R) == 4) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(mesh) + node);
                acc[0] = fmaf(w, v.x, acc[0]);
                acc[1] = fmaf(w, v.y, acc[1]);
                acc[2] = fmaf(w, v.z, acc[2]);
                acc[3] = fmaf(w, v.w, acc[3]);
            } else {
                const V *mp = mesh + node * C;
                for (int c = 0; c < C; ++c) acc[c] = fma(w, load_val<V, R>(mp + c), acc[c]);
            }
        }
        if constexpr (CT == 4 && sizeof(V) == 4 && sizeof(R) == 4)
            __stcs(reinterpret_cast<float4 *>(vals) + m, make_float4(acc[0], acc[1], acc[2], acc[3]));
        else
            for (int c = 0; c < C; ++c) store_val<V, R>(vals + m * C + c, acc[c]);
    }
}

cudaError_t launch_m2p_quadratic(int n, long long N, const void *pos, pfem_dtype pos_t, int C,
                                 const void *mesh, void *vals, pfem_dtype val_t, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    const MQTable &T = mq_table();
    long long blocks = (N + 255) / 256;
    if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
    const bool aligned = ((reinterpret_cast<uintptr_t>(mesh) | reinterpret_cast<uintptr_t>(vals)) & 15) == 0;
    if (val_t == PFEM_F64 && pos_t == PFEM_F64)
        k_m2p_q<double, double, double, 0><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const double *)pos, C, (const double *)mesh, (double *)vals, T);
    else if (val_t == PFEM_F32 && pos_t == PFEM_F32 && C == 4 && aligned)
        k_m2p_q<float, float, float, 4><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const float *)pos, C, (const float *)mesh, (float *)vals, T);
    else if (val_t == PFEM_F32 && pos_t == PFEM_F32)
        k_m2p_q<float, float, float, 0><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const float *)pos, C, (const float *)mesh, (float *)vals, T);
    else if (val_t == PFEM_BF16 && pos_t == PFEM_F32)
        k_m2p_q<float, __nv_bfloat16, float, 0><<<(unsigned)blocks, 256, 0, s>>>(n, N, (const float *)pos, C, (const __nv_bfloat16 *)mesh, (__nv_bfloat16 *)vals, T);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

}  // namespace pfem
