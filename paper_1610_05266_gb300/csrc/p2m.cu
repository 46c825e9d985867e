// p2m.cu -- launchers of the particle-to-mesh kernels (fused apply, explicit weights, apply
// from explicit weights) and of the Delaunay-star diagnostic.
#include <algorithm>
#include <climits>

#include "internal.h"
#include "p2m_tiled.cuh"

namespace pfem {

// The queue of nodes for the FP64 SVD pass lives in the workspace after the 256-byte status
// block: a counter at byte 256, node indices from byte 512.  A workspace of 256 bytes has no
// queue (such nodes then report PFEM_ERR_DEGENERATE).
static void set_queue(P2MArgs &a, void *ws, size_t ws_bytes)
{
    const long long nodes = (long long)a.n * a.n;
    const long long cap = ws_bytes >= 520 ? (long long)((ws_bytes - 512) / sizeof(long long)) : 0;
    a.defer_cap = (int)std::min(std::min(cap, nodes), (long long)INT_MAX);
    a.defer_count = a.defer_cap > 0 ? (int *)((char *)ws + 256) : nullptr;
    a.defer_list = a.defer_cap > 0 ? (long long *)((char *)ws + 512) : nullptr;
}

static P2MArgs make_args(const GeoArgs &g, DevStatus *st)
{
    P2MArgs a;
    a.n = g.n;
    a.B.q = (const uint2 *)g.q_sorted;
    a.B.start = g.cell_start;
    a.B.nb = g.nb;
    a.B.rmax = g.rmax;
    a.B.dmax = g.dmax;
    a.R0 = g.R0;
    a.pos = g.pos_sorted;
    a.perm = nullptr;
    a.vals = nullptr;
    a.C = 0;
    a.out = nullptr;
    a.w_idx = nullptr;
    a.w = nullptr;
    a.K = 0;
    a.status = st;
    return a;
}

static dim3 node_grid(int n) { return dim3((n + 15) / 16, (n + 7) / 8); }

// Nodes per tile side for the tiled kernel (0: use the per-thread kernel): the staged window
// (tile bins + halo) must fit the shared-memory capacity and stay within half the torus.
int tile_side(int n, int nb, long long N)
{
    const double bins_per_cell = (double)nb / (double)(n - 1);
    const double ppb = (double)N / ((double)nb * nb);
    for (int T = 16; T >= 4; T >>= 1) {
        const int w = (int)ceil((T - 1) * bins_per_cell) + 2 + 2 * THB;
        if (w * w <= TMAXB && 2 * w <= nb && w * w * ppb * 1.1 <= TMAXP) return T;
    }
    return 0;
}

template <typename P, typename V, typename R, typename S, bool REF, int SHAPE, bool W>
static cudaError_t go_fast(const P2MArgs &a, cudaStream_t s, int T)
{
    if (!W && T > 0) {
        auto k = k_p2m_tiled<P, V, R, S, REF, SHAPE>;
        const int bytes = (int)sizeof(TileSmem);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        const int tx = (a.n + T - 1) / T;
        k<<<tx * tx, TT, bytes, s>>>(a, T, tx);
        count_launch();
        return cudaGetLastError();
    }
    k_p2m<P, V, R, S, REF, SHAPE, W><<<node_grid(a.n), 128, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout of quadratic P2M after the 256-byte status block: the queue counter at 256,
// the queue from 512 (8 bytes per node), then the node records of the two-kernel path.
static size_t recs_offset(long long nodes) { return al256(512 + 8 * (size_t)nodes); }

size_t p2m_ws_bytes(long long nodes)
{
    NodeRecs r;
    return recs_offset(nodes) + node_recs_layout(nullptr, nodes, &r);
}

static bool set_recs(NodeRecs &r, void *ws, size_t ws_bytes, long long nodes)
{
    if (ws_bytes < p2m_ws_bytes(nodes)) return false;
    node_recs_layout((char *)ws + recs_offset(nodes), nodes, &r);
    return true;
}

// Fused P2M: the fast pass over all nodes (one kernel, or with node records and FP32 solves
// the geometry and solve kernels), then (quadratic shape functions, with a queue) the FP64 SVD pass over the
// nodes it queued.
template <typename P, typename V, typename R, typename S, bool REF, int SHAPE, bool W>
static cudaError_t go(const P2MArgs &a, cudaStream_t s, int T = 0, const NodeRecs *rec = nullptr)
{
    const bool queue = SHAPE == PFEM_SHAPE_QUADRATIC && a.defer_cap > 0;
    if (queue) {
        cudaError_t e = cudaMemsetAsync(a.defer_count, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e;
    if (SHAPE == PFEM_SHAPE_QUADRATIC && !W && T == 0 && rec && sizeof(S) == sizeof(float)) {
        k_p2m_geom<P, V, R><<<node_grid(a.n), 128, 0, s>>>(a, *rec);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_p2m_solve<P, V, R, S, REF><<<(unsigned)((rec->nodes + 127) / 128), 128, 0, s>>>(a, *rec);
        count_launch();
        e = cudaGetLastError();
    } else {
        e = go_fast<P, V, R, S, REF, SHAPE, W>(a, s, T);
    }
    if (e != cudaSuccess || !queue) return e;
    k_p2m_fix<P, V, R, W><<<152, 128, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_p2m(const GeoArgs &g, const int *perm, int C, const void *vals,
                       pfem_dtype val_t, pfem_shape shape, pfem_solve solve, void *out,
                       DevStatus *st, size_t ws_bytes, cudaStream_t s)
{
    P2MArgs a = make_args(g, st);
    set_queue(a, st, ws_bytes);
    a.perm = perm;
    a.vals = vals;
    a.C = C;
    a.out = out;
    const bool q = shape == PFEM_SHAPE_QUADRATIC;
    const int T = g.tiled ? tile_side(g.n, g.nb, g.N) : 0;
    NodeRecs recs;
    const NodeRecs *r = set_recs(recs, st, ws_bytes, (long long)g.n * g.n) ? &recs : nullptr;
    if (val_t == PFEM_F64) {   // positions FP64, arithmetic FP64
        if (!q) return go<double, double, double, double, false, 0, false>(a, s, T);
        return go<double, double, double, double, false, 1, false>(a, s, T, r);
    }
    if (val_t == PFEM_F32) {   // positions FP32, arithmetic FP32
        if (!q) return go<float, float, float, float, false, 0, false>(a, s, T);
        if (solve == PFEM_SOLVE_F64) return go<float, float, float, double, false, 1, false>(a, s, T, r);
        if (solve == PFEM_SOLVE_F32) return go<float, float, float, float, false, 1, false>(a, s, T, r);
        return go<float, float, float, float, true, 1, false>(a, s, T, r);
    }
    if (!q) return go<float, __nv_bfloat16, float, float, false, 0, false>(a, s, T);
    if (solve == PFEM_SOLVE_F64) return go<float, __nv_bfloat16, float, double, false, 1, false>(a, s, T, r);
    if (solve == PFEM_SOLVE_F32) return go<float, __nv_bfloat16, float, float, false, 1, false>(a, s, T, r);
    return go<float, __nv_bfloat16, float, float, true, 1, false>(a, s, T, r);
}

cudaError_t launch_shape(const GeoArgs &g, pfem_shape shape, pfem_solve solve, int K, int *w_idx,
                         void *w, pfem_dtype w_t, DevStatus *st, size_t ws_bytes, cudaStream_t s)
{
    P2MArgs a = make_args(g, st);
    set_queue(a, st, ws_bytes);
    a.K = K;
    a.w_idx = w_idx;
    a.w = w;
    const bool q = shape == PFEM_SHAPE_QUADRATIC;
    if (w_t == PFEM_F64) {
        if (!q) return go<double, double, double, double, false, 0, true>(a, s);
        return go<double, double, double, double, false, 1, true>(a, s);
    }
    if (!q) return go<float, float, float, float, false, 0, true>(a, s);
    if (solve == PFEM_SOLVE_F64) return go<float, float, float, double, false, 1, true>(a, s);
    if (solve == PFEM_SOLVE_F32) return go<float, float, float, float, false, 1, true>(a, s);
    return go<float, float, float, float, true, 1, true>(a, s);
}

// alpha_i = sum_k w[i,k] alpha[w_idx[i,k]] (explicit-weight P2M)
template <typename V, typename R>
__global__ void __launch_bounds__(256) k_apply(long long nodes, int K, const int *__restrict__ w_idx,
                                               const R *__restrict__ w, const int *__restrict__ perm,
                                               int C, const V *__restrict__ vals, V *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        R acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = R(0);
        for (int k = 0; k < K; ++k) {
            const int s = __ldg(w_idx + i * K + k);
            if (s < 0) break;
            const R wk = __ldg(w + i * K + k);
            R v[8];
            load_vals<V, R>(vals, perm, s, C, v);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < C) acc[c] = fma(wk, v[c], acc[c]);
        }
        store_vals<V, R>(out, i, C, acc);
    }
}

cudaError_t launch_apply(int n, const int *perm, int C, const void *vals, pfem_dtype val_t,
                         const int *w_idx, const void *w, int K, pfem_dtype w_t, void *out,
                         cudaStream_t s)
{
    const long long nodes = (long long)n * n;
    long long blocks = (nodes + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (val_t == PFEM_F64 && w_t == PFEM_F64)
        k_apply<double, double><<<(unsigned)blocks, 256, 0, s>>>(
            nodes, K, w_idx, (const double *)w, perm, C, (const double *)vals, (double *)out);
    else if (val_t == PFEM_F32 && w_t == PFEM_F32)
        k_apply<float, float><<<(unsigned)blocks, 256, 0, s>>>(
            nodes, K, w_idx, (const float *)w, perm, C, (const float *)vals, (float *)out);
    else if (val_t == PFEM_BF16 && w_t == PFEM_F32)
        k_apply<__nv_bfloat16, float><<<(unsigned)blocks, 256, 0, s>>>(
            nodes, K, w_idx, (const float *)w, perm, C, (const __nv_bfloat16 *)vals,
            (__nv_bfloat16 *)out);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(128, PFEM_P2M_MIN_BLOCKS) k_stars(Bins B, int R0, long long N, int *nbrs, int *counts,
                                               DevStatus *st)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        int loc[KMAX];
        const int c = star_of(B, (int)v, R0, loc);
        if (c < 0) record_error(st, -c, v);
        const int cnt = c < 0 ? 0 : c;
        for (int k = 0; k < KMAX; ++k) nbrs[v * KMAX + k] = k < cnt ? loc[k] : -1;
        counts[v] = cnt;
    }
}

cudaError_t launch_stars(const GeoArgs &g, int *nbrs, int *counts, DevStatus *st, cudaStream_t s)
{
    P2MArgs a = make_args(g, st);
    long long blocks = (g.N + 127) / 128;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    if (blocks < 1) blocks = 1;
    k_stars<<<(unsigned)blocks, 128, 0, s>>>(a.B, g.R0, g.N, nbrs, counts, st);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pfem
