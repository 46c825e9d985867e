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
    if (blocks > 152LL * 16) blocks = 152LL * 16;
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
        if (blocks > 152LL * 16) blocks = 152LL * 16;
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

}  // namespace pfem
