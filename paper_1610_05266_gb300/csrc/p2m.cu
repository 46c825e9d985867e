// p2m.cu -- launchers of the particle-to-mesh kernels (fused apply, explicit weights, apply
// from explicit weights) and of the Delaunay-star diagnostic.
#include <algorithm>
#include <climits>

#include "internal.h"
#include "p2m.cuh"

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
    a.B.kcap = g.kcap;
    a.B.walk_cap = g.walk_cap;
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
    a.ucap = g.ucap;
    return a;
}

static dim3 node_grid(int n) { return dim3((n + 15) / 16, (n + 7) / 8); }

// The table path's fast pass as one kernel (k_p2m_tab) or as the geometry and solve kernels with
// node records in between.  Measured at 1025^2 nodes / 2048^2 particles (geometry + solve):
// FP64-residual refinement 1.21 -> 1.07 ms fused, plain FP32 0.58 -> 0.53 ms, float-float
// refinement 0.84 -> 0.89 ms; the float-float solve keeps the two kernels.
#ifndef PFEM_P2M_FUSED_TAB
#define PFEM_P2M_FUSED_TAB 1
#endif

template <typename P, typename V, typename R, typename S, int REF, int SHAPE, bool W>
static cudaError_t go_fast(const P2MArgs &a, cudaStream_t s)
{
    k_p2m<P, V, R, S, REF, SHAPE, W><<<node_grid(a.n), 128, 0, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout of P2M after the 256-byte status block: the fix-pass queue counter at byte
// 256 and the star-table queue counter at byte 260, the fix-pass queue from byte 512 (8 bytes
// per node), then the node records and the star table of the table path.
static size_t recs_offset(long long nodes) { return al256(512 + 8 * (size_t)nodes); }

size_t p2m_ws_bytes(long long nodes, long long N)
{
    NodeRecs r;
    const size_t recs = al256(node_recs_layout(nullptr, nodes, &r));
    return recs_offset(nodes) + recs + star_tab_bytes(N);
}

// Records and star table in ws, when it has room for them.
static bool set_table(NodeRecs &r, StarTab &t, void *ws, size_t ws_bytes, long long nodes,
                      long long N)
{
    if (ws_bytes < p2m_ws_bytes(nodes, N)) return false;
    char *base = (char *)ws + recs_offset(nodes);
    const size_t recs = al256(node_recs_layout(base, nodes, &r));
    t = star_tab_layout(base + recs, N, (int *)((char *)ws + 260));
    return true;
}

// P2M: the fast pass over all nodes, then the fix pass over the nodes it queued.  With quadratic
// shape functions, the apply form and room for the table, the fast pass is the star table and
// then k_p2m_tab (location, edge solves and apply per node), or, for the float-float solve, the
// geometry kernel (node records) and the solve kernel; otherwise one kernel that searches the
// stars per node.
// Stage events (when the caller's context has them): 0 before the fast pass, 1 after the star
// table, 2 after the geometry kernel (right before k_p2m_tab), 3 after the solve kernel (after
// k_p2m_tab), 4 after the fix pass.
template <typename P, typename V, typename R, typename S, int REF, int SHAPE, bool W>
static cudaError_t go(const GeoArgs &g, const P2MArgs &a, cudaStream_t s,
                      const NodeRecs *rec = nullptr, const StarTab *tab = nullptr)
{
    const int R0 = g.R0, rmax_far = g.rmax_far;
    cudaError_t e;
    stage_event(g, 0, s);
    if (a.defer_cap > 0) {
        e = cudaMemsetAsync(a.defer_count, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
    }
    if (SHAPE == PFEM_SHAPE_QUADRATIC && !W && rec && tab) {
        e = launch_star_table(a.B, R0, rmax_far, *tab, a.status, s);
        if (e != cudaSuccess) return e;
        stage_event(g, 1, s);
#if PFEM_P2M_FUSED_TAB
        if (!W && REF != REFINE_FF) {
            stage_event(g, 2, s);
            e = wait_values(g, s);
            if (e != cudaSuccess) return e;
            k_p2m_tab<P, V, R, S, REF><<<node_grid(a.n), 128, 0, s>>>(a, *tab);
            count_launch();
            e = cudaGetLastError();
            stage_event(g, 3, s);
        } else
#endif
        {
        k_p2m_geom<P, V, R><<<node_grid(a.n), 128, 0, s>>>(a, *tab, *rec);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        stage_event(g, 2, s);
        if (!W) {
            e = wait_values(g, s);
            if (e != cudaSuccess) return e;
        }
        k_p2m_solve<P, V, R, S, REF><<<(unsigned)((rec->nodes + 127) / 128), 128, 0, s>>>(a, *rec);
        count_launch();
        e = cudaGetLastError();
        stage_event(g, 3, s);
        }
    } else {
        if (!W) {
            e = wait_values(g, s);
            if (e != cudaSuccess) return e;
        }
        e = go_fast<P, V, R, S, REF, SHAPE, W>(a, s);
    }
    if (e != cudaSuccess || a.defer_cap <= 0) return e;
    P2MArgs f = a;
    f.B.rmax = rmax_far > a.B.rmax ? rmax_far : a.B.rmax;
    if (SHAPE == PFEM_SHAPE_QUADRATIC && !W && rec && tab)
        k_p2m_fix_tab<P, V, R, sizeof(S) == 4><<<num_sms(), 128, 0, s>>>(f, *tab);
    else
        k_p2m_fix<P, V, R, SHAPE, W><<<num_sms(), 128, 0, s>>>(f);
    count_launch();
    stage_event(g, 4, s);
    return cudaGetLastError();
}

// Compute type S and refinement of each solve for FP32 arithmetic.
template <typename P, typename V, int SHAPE, bool W>
static cudaError_t go_solve(pfem_solve solve, const GeoArgs &g, const P2MArgs &a, cudaStream_t s,
                            const NodeRecs *r, const StarTab *t)
{
    switch (solve) {
    case PFEM_SOLVE_F64: return go<P, V, float, double, REFINE_NONE, SHAPE, W>(g, a, s, r, t);
    case PFEM_SOLVE_F32: return go<P, V, float, float, REFINE_NONE, SHAPE, W>(g, a, s, r, t);
    case PFEM_SOLVE_F32_REFINED: return go<P, V, float, float, REFINE_F64, SHAPE, W>(g, a, s, r, t);
    default: return go<P, V, float, float, REFINE_FF, SHAPE, W>(g, a, s, r, t);
    }
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
    NodeRecs recs;
    StarTab tab;
    const bool table = set_table(recs, tab, st, ws_bytes, (long long)g.n * g.n, g.N);
    const NodeRecs *r = table ? &recs : nullptr;
    const StarTab *t = table ? &tab : nullptr;
    if (val_t == PFEM_F64) {   // positions FP64, arithmetic FP64
        if (!q) return go<double, double, double, double, REFINE_NONE, 0, false>(g, a, s);
        return go<double, double, double, double, REFINE_NONE, 1, false>(g, a, s, r, t);
    }
    if (val_t == PFEM_F32) {   // positions FP32, arithmetic FP32
        if (!q) return go<float, float, float, float, REFINE_NONE, 0, false>(g, a, s);
        return go_solve<float, float, 1, false>(solve, g, a, s, r, t);
    }
    if (!q) return go<float, __nv_bfloat16, float, float, REFINE_NONE, 0, false>(g, a, s);
    return go_solve<float, __nv_bfloat16, 1, false>(solve, g, a, s, r, t);
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
        if (!q) return go<double, double, double, double, REFINE_NONE, 0, true>(g, a, s);
        return go<double, double, double, double, REFINE_NONE, 1, true>(g, a, s);
    }
    if (!q) return go<float, float, float, float, REFINE_NONE, 0, true>(g, a, s);
    return go_solve<float, float, 1, true>(solve, g, a, s, nullptr, nullptr);
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
    if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
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

// The star table written straight into the caller's arrays, then padded: unused entries -1 and
// a failed star's count 0 (its error is in the status word).
__global__ void k_stars_pad(long long N, int *nbrs, int *counts)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const int w = (int)((unsigned)counts[v] & 255u) - 128;   // drop the table's stamp
        const int c = w < 0 ? 0 : w;
        for (int k = c; k < KMAX; ++k) nbrs[v * KMAX + k] = -1;
        counts[v] = c;
    }
}

// Workspace bytes of pfem_delaunay_stars: the status block and the retry queue.
size_t stars_ws_bytes(long long N) { return 256 + 4 * (size_t)(N > 0 ? N : 1); }

cudaError_t launch_stars(const GeoArgs &g, int *nbrs, int *counts, DevStatus *st, cudaStream_t s)
{
    P2MArgs a = make_args(g, st);
    StarTab t;
    t.nbr = nbrs;
    t.cnt = counts;
    t.queue = (int *)((char *)st + 256);
    t.qcount = (int *)((char *)st + 64);
    t.N = g.N;
    t.gen = next_tab_gen();
    cudaError_t e = launch_star_table(a.B, g.R0, g.rmax_far, t, st, s);
    if (e != cudaSuccess) return e;
    long long blocks = (g.N + 255) / 256;
    if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
    if (blocks < 1) blocks = 1;
    k_stars_pad<<<(unsigned)blocks, 256, 0, s>>>(g.N, nbrs, counts);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pfem
