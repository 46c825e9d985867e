// capi.cu -- the extern "C" entry points declared in include/pfem.h: argument checks,
// workspace layout and dispatch to the kernels.  No entry point allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.h"

using namespace pfem;

#include <atomic>

namespace pfem {

static std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Binning scratch for nb*nb bins and N particles; with a mesh (n > 0) the total also covers
// what quadratic P2M keeps in the workspace once the cells are built (the queue of nodes for
// the SVD pass and the per-node records of the two-kernel path).
WsLayout ws_layout(int n, int nb, long long N, int C)
{
    (void)C;
    WsLayout L = ws_layout_bins((long long)nb * nb, N);
    if (n > 0) L.total = std::max(L.total, p2m_ws_bytes((long long)n * n));
    return L;
}

WsLayout ws_layout_bins(long long nbins, long long N)
{
    WsLayout L;
    size_t off = 0;
    L.status = off;
    off += 256;
    L.count = off;
    off = align256(off + sizeof(int) * (size_t)(nbins + 1));
    L.key = off;
    off = align256(off + sizeof(int) * (size_t)(N > 0 ? N : 1));
    L.rank = off;
    off = align256(off + sizeof(int) * (size_t)(N > 0 ? N : 1));
    L.scan = off;
    off = align256(off + sizeof(int) * scan_scratch_ints(nbins + 1));
    L.bwd = off;
    L.total = off;
    return L;
}

}  // namespace pfem

static pfem_status from_cuda(cudaError_t e) { return e == cudaSuccess ? PFEM_OK : PFEM_ERR_CUDA; }

static bool geom_ok(int32_t n, int32_t nb, int64_t N)
{
    return n >= 9 && nb >= 8 && (long long)nb * nb < (1LL << 30) && N >= 3 && N < (1LL << 31) &&
           (long long)n * n < (1LL << 40);
}

// First search radius (bins) and the largest one tried: the first region reaches about 1.2
// mean particle spacings beyond the particle's own bin; regions stay within a quarter of the
// torus so that signed 32-bit fixed-point differences never alias.
static void radii(int32_t nb, int64_t N, int *R0, int *rmax)
{
    const double h_over_bw = (double)nb / std::sqrt((double)N);
    int r = (int)std::ceil(1.2 * h_over_bw);
    if (r < 1) r = 1;
    int rm = r + 3;
    if (rm > nb / 4 - 1) rm = nb / 4 - 1;
    *R0 = r;
    *rmax = rm;
}

namespace pfem {
void radii_for(int nb, long long N, int *R0, int *rmax, float *dmax)
{
    radii(nb, N, R0, rmax);
    *dmax = (float)std::fmin(2.0 * 4294967296.0 / std::sqrt((double)N), 1073741824.0);
}
}  // namespace pfem

static bool make_geo(int32_t n, int32_t nb, int64_t N, const void *pos_sorted, pfem_dtype pos_t,
                     const uint32_t *q_sorted, const int32_t *cell_start, GeoArgs *g)
{
    if (!geom_ok(n, nb, N) || !pos_sorted || !q_sorted || !cell_start) return false;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return false;
    g->n = n;
    g->nb = nb;
    g->N = N;
    g->pos_sorted = pos_sorted;
    g->pos_t = pos_t;
    g->q_sorted = q_sorted;
    g->cell_start = cell_start;
    // first search radius, largest radius, and the distance cutoff of the first star attempt
    // (2.0 mean particle spacings, fixed point: above the largest Delaunay circumdiameter of
    // jittered lattices at jitter 0.25, 1.97 spacings; a star that fails it takes the region search)
    radii_for(nb, N, &g->R0, &g->rmax, &g->dmax);
    // The shared-memory tiled P2M is opt-in: on the jittered-lattice workloads it measured
    // slower than the per-thread kernel (the cost is in the divergent star search, not memory).
    g->tiled = getenv("PFEM_TILED") != nullptr;
    return g->rmax >= g->R0;
}

extern "C" {

int pfem_abi_version(void) { return 1; }

uint64_t pfem_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

const char *pfem_status_string(pfem_status s)
{
    switch (s) {
    case PFEM_OK: return "ok";
    case PFEM_ERR_INVALID_ARG: return "invalid argument";
    case PFEM_ERR_CUDA: return "CUDA error";
    case PFEM_ERR_WORKSPACE: return "workspace too small";
    case PFEM_ERR_CAPACITY: return "capacity exceeded";
    case PFEM_ERR_DEGENERATE: return "degenerate input";
    case PFEM_ERR_TIMEOUT: return "iteration cap reached";
    }
    return "unknown status";
}

int32_t pfem_default_bins(int32_t n, int64_t N)
{
    (void)n;
    long long nb = (long long)std::llround(std::sqrt((double)(N > 0 ? N : 1) / 4.0));
    if (nb < 8) nb = 8;
    if (nb > 16384) nb = 16384;
    return (int32_t)nb;
}

size_t pfem_workspace_size(int32_t n, int32_t nb, int64_t N, int32_t C)
{
    if (nb < 1 || N < 0) return 0;
    return ws_layout(n, nb, N, C).total;
}

pfem_status pfem_read_status(const void *ws, int32_t *status_host, int64_t *detail_host,
                             void *stream)
{
    if (!ws || !status_host) return PFEM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus h;
    cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return PFEM_ERR_CUDA;
    *status_host = h.code;
    if (detail_host) *detail_host = h.code ? h.detail : -1;
    return PFEM_OK;
}

pfem_status pfem_reset_status(void *ws, void *stream)
{
    if (!ws) return PFEM_ERR_INVALID_ARG;
    return from_cuda(cudaMemsetAsync(ws, 0, sizeof(DevStatus), (cudaStream_t)stream));
}

pfem_status pfem_build_cells(int32_t nb, int64_t N, const void *pos, pfem_dtype pos_t,
                             int32_t *cell_start, int32_t *perm, void *pos_sorted,
                             uint32_t *q_sorted, void *ws, size_t ws_bytes, void *stream)
{
    if (nb < 1 || (long long)nb * nb >= (1LL << 30) || N < 0 || N >= (1LL << 31)) return PFEM_ERR_INVALID_ARG;
    if (!cell_start || !ws || (N > 0 && (!pos || !perm || !pos_sorted || !q_sorted)))
        return PFEM_ERR_INVALID_ARG;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    const WsLayout L = ws_layout(0, nb, N, 1);
    if (ws_bytes < L.total) return PFEM_ERR_WORKSPACE;
    return from_cuda(launch_build_cells(nb, N, pos, pos_t, cell_start, perm, pos_sorted, q_sorted,
                                        L, ws, (cudaStream_t)stream));
}

pfem_status pfem_delaunay_stars(int32_t nb, int64_t N, const uint32_t *q_sorted,
                                const int32_t *cell_start, int32_t *nbrs, int32_t *counts,
                                void *ws, size_t ws_bytes, void *stream)
{
    GeoArgs g;
    if (!make_geo(9, nb, N, q_sorted, PFEM_F32, q_sorted, cell_start, &g) || !nbrs || !counts || !ws)
        return PFEM_ERR_INVALID_ARG;
    if (ws_bytes < 256) return PFEM_ERR_WORKSPACE;
    return from_cuda(launch_stars(g, nbrs, counts, (DevStatus *)ws, (cudaStream_t)stream));
}

pfem_status pfem_shape_quadratic(int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                                 pfem_dtype pos_t, const uint32_t *q_sorted,
                                 const int32_t *cell_start, pfem_shape shape, pfem_solve solve,
                                 int32_t K, int32_t *w_idx, void *w, pfem_dtype w_t, void *ws,
                                 size_t ws_bytes, void *stream)
{
    GeoArgs g;
    if (!make_geo(n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g)) return PFEM_ERR_INVALID_ARG;
    if (!w_idx || !w || !ws || K < 3 || K > PFEM_KW_MAX) return PFEM_ERR_INVALID_ARG;
    if (shape != PFEM_SHAPE_LINEAR && shape != PFEM_SHAPE_QUADRATIC) return PFEM_ERR_INVALID_ARG;
    if (solve < PFEM_SOLVE_F64 || solve > PFEM_SOLVE_F32_REFINED) return PFEM_ERR_INVALID_ARG;
    // FP64 weights come from FP64 positions with the FP64 solve; FP32 weights from FP32 positions
    if (w_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)) return PFEM_ERR_INVALID_ARG;
    if (w_t == PFEM_F32 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    if (w_t == PFEM_BF16) return PFEM_ERR_INVALID_ARG;
    if (ws_bytes < 256) return PFEM_ERR_WORKSPACE;
    return from_cuda(launch_shape(g, shape, solve, K, w_idx, w, w_t, (DevStatus *)ws, ws_bytes,
                                  (cudaStream_t)stream));
}

pfem_status pfem_project_p2m(int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                             pfem_dtype pos_t, const uint32_t *q_sorted,
                             const int32_t *cell_start, const int32_t *perm, int32_t C,
                             const void *vals, pfem_dtype val_t, pfem_shape shape,
                             pfem_solve solve, const int32_t *w_idx, const void *w, int32_t K,
                             pfem_dtype w_t, void *mesh_vals, void *ws, size_t ws_bytes,
                             void *stream)
{
    GeoArgs g;
    if (!make_geo(n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g)) return PFEM_ERR_INVALID_ARG;
    if (C < 1 || C > 8 || !vals || !mesh_vals || !ws) return PFEM_ERR_INVALID_ARG;
    if (val_t != PFEM_F64 && val_t != PFEM_F32 && val_t != PFEM_BF16) return PFEM_ERR_INVALID_ARG;
    if (ws_bytes < 256) return PFEM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (w_idx || w) {
        if (!w_idx || !w || K < 3 || K > PFEM_KW_MAX) return PFEM_ERR_INVALID_ARG;
        if (!((val_t == PFEM_F64 && w_t == PFEM_F64) || (val_t != PFEM_F64 && w_t == PFEM_F32)))
            return PFEM_ERR_INVALID_ARG;
        return from_cuda(launch_apply(n, perm, C, vals, val_t, w_idx, w, K, w_t, mesh_vals, s));
    }
    if (shape != PFEM_SHAPE_LINEAR && shape != PFEM_SHAPE_QUADRATIC) return PFEM_ERR_INVALID_ARG;
    if (solve < PFEM_SOLVE_F64 || solve > PFEM_SOLVE_F32_REFINED) return PFEM_ERR_INVALID_ARG;
    // FP64 values use FP64 positions and the FP64 solve; FP32/BF16 values use FP32 positions
    if (val_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)) return PFEM_ERR_INVALID_ARG;
    if (val_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_p2m(g, perm, C, vals, val_t, shape, solve, mesh_vals, (DevStatus *)ws,
                                ws_bytes, s));
}

pfem_status pfem_interp_m2p(int32_t n, int64_t N, const void *pos, pfem_dtype pos_t, int32_t C,
                            const void *mesh_vals, void *vals, pfem_dtype val_t, void *stream)
{
    if (n < 9 || N < 0 || N >= (1LL << 40) || C < 1 || C > 8) return PFEM_ERR_INVALID_ARG;
    if (N > 0 && (!pos || !mesh_vals || !vals)) return PFEM_ERR_INVALID_ARG;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    if (val_t != PFEM_F64 && val_t != PFEM_F32 && val_t != PFEM_BF16) return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_m2p(n, N, pos, pos_t, C, mesh_vals, vals, val_t, (cudaStream_t)stream));
}

size_t pfem_backward_workspace_size(int32_t n, int64_t N, int32_t K)
{
    if (n < 1 || N < 0 || K < 0) return 0;
    return bwd_layout(n, N, K).total;
}

pfem_status pfem_interp_m2p_quadratic(int32_t n, int64_t N, const void *pos, pfem_dtype pos_t,
                                      int32_t C, const void *mesh_vals, void *vals,
                                      pfem_dtype val_t, void *stream)
{
    if (n < 9 || N < 0 || N >= (1LL << 40) || C < 1 || C > 8) return PFEM_ERR_INVALID_ARG;
    if (N > 0 && (!pos || !mesh_vals || !vals)) return PFEM_ERR_INVALID_ARG;
    if (!((val_t == PFEM_F64 && pos_t == PFEM_F64) || (val_t != PFEM_F64 && pos_t == PFEM_F32)))
        return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_m2p_quadratic(n, N, pos, pos_t, C, mesh_vals, vals, val_t,
                                          (cudaStream_t)stream));
}

pfem_status pfem_project_backward(int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                                  pfem_dtype pos_t, const uint32_t *q_sorted,
                                  const int32_t *cell_start, const int32_t *perm, int32_t C,
                                  const void *vals, pfem_dtype val_t, pfem_shape shape,
                                  pfem_solve solve, pfem_backward_mode mode,
                                  const int32_t *w_idx, const void *w, int32_t K,
                                  pfem_dtype w_t, const void *grad_mesh, void *grad_vals,
                                  void *grad_pos, void *ws, size_t ws_bytes, void *stream)
{
    GeoArgs g;
    if (!make_geo(n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g)) return PFEM_ERR_INVALID_ARG;
    if (C < 1 || C > 8 || !vals || !grad_mesh || !grad_vals || !ws) return PFEM_ERR_INVALID_ARG;
    if (shape != PFEM_SHAPE_LINEAR && shape != PFEM_SHAPE_QUADRATIC) return PFEM_ERR_INVALID_ARG;
    if (val_t == PFEM_F64) {
        if (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64) return PFEM_ERR_INVALID_ARG;
    } else if (val_t == PFEM_F32) {
        if (pos_t != PFEM_F32 || (solve != PFEM_SOLVE_F64 && solve != PFEM_SOLVE_F32))
            return PFEM_ERR_INVALID_ARG;
    } else {
        return PFEM_ERR_INVALID_ARG;
    }
    const bool ckpt = mode == PFEM_BACKWARD_CHECKPOINT;
    if (mode != PFEM_BACKWARD_RECOMPUTE && !ckpt) return PFEM_ERR_INVALID_ARG;
    if (ckpt) {
        if (!w_idx || !w || K < 3 || K > PFEM_KW_MAX) return PFEM_ERR_INVALID_ARG;
        if (w_t != val_t) return PFEM_ERR_INVALID_ARG;
    }
    const BwdLayout L = bwd_layout(n, N, ckpt ? K : 0);
    if (ws_bytes < L.total) return PFEM_ERR_WORKSPACE;
    return from_cuda(launch_p2m_backward(g, perm, C, vals, val_t, shape, solve, ckpt, w_idx, w,
                                         ckpt ? K : 0, grad_mesh, grad_vals, grad_pos, L, ws,
                                         (cudaStream_t)stream));
}

pfem_status pfem_interp_m2p_backward(int32_t n, int32_t nb, int64_t N, const void *pos,
                                     pfem_dtype pos_t, const int32_t *cell_start,
                                     const int32_t *perm, int32_t C, const void *mesh_vals,
                                     const void *grad_vals, pfem_dtype val_t, void *grad_mesh,
                                     void *grad_pos, void *stream)
{
    if (n < 9 || nb < 1 || (long long)nb * nb >= (1LL << 30) || N < 0 || N >= (1LL << 31) ||
        C < 1 || C > 8)
        return PFEM_ERR_INVALID_ARG;
    if (!cell_start || !grad_mesh || (N > 0 && (!pos || !perm || !grad_vals)) ||
        (grad_pos && !mesh_vals))
        return PFEM_ERR_INVALID_ARG;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    if (val_t != PFEM_F64 && val_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_m2p_backward(n, nb, N, pos, pos_t, cell_start, perm, C, mesh_vals,
                                         grad_vals, val_t, grad_mesh, grad_pos,
                                         (cudaStream_t)stream));
}

size_t pfem_batch_plan_size(int32_t P)
{
    return P < 1 ? 0 : batch_plan_bytes(P);
}

pfem_status pfem_batch_plan_init(int32_t P, const pfem_batch_problem *problems, void *plan,
                                 int64_t *totals)
{
    if (P < 1 || !problems || !plan || !totals) return PFEM_ERR_INVALID_ARG;
    long long Nt = 0, bt = 0, nt = 0;
    const int st = batch_plan_build(P, problems, plan, &Nt, &bt, &nt);
    if (st != PFEM_OK) return (pfem_status)st;
    totals[0] = Nt;
    totals[1] = bt;
    totals[2] = nt;
    return PFEM_OK;
}

size_t pfem_batch_workspace_size(int64_t N_total, int64_t bins_total, int64_t nodes_total)
{
    if (N_total < 0 || bins_total < 1 || nodes_total < 0) return 0;
    const size_t b = ws_layout_bins(bins_total, N_total).total;
    return nodes_total > 0 ? std::max(b, batch_p2m_ws_bytes(nodes_total)) : b;
}

pfem_status pfem_batch_build_cells(const void *plan, int64_t N_total, int64_t bins_total,
                                   const void *pos, pfem_dtype pos_t, int32_t *cell_start,
                                   int32_t *perm, void *pos_sorted, uint32_t *q_sorted, void *ws,
                                   size_t ws_bytes, void *stream)
{
    if (!plan || !pos || !cell_start || !perm || !pos_sorted || !q_sorted || !ws) return PFEM_ERR_INVALID_ARG;
    if (N_total < 1 || N_total >= (1LL << 31) || bins_total < 1 || bins_total >= (1LL << 31)) return PFEM_ERR_INVALID_ARG;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    const WsLayout L = ws_layout_bins(bins_total, N_total);
    if (ws_bytes < L.total) return PFEM_ERR_WORKSPACE;
    return from_cuda(launch_batch_build_cells(plan, N_total, bins_total, pos, pos_t, cell_start, perm,
                                              pos_sorted, q_sorted, L, ws, (cudaStream_t)stream));
}

pfem_status pfem_batch_project_p2m(const void *plan, int64_t nodes_total, const void *pos_sorted,
                                   pfem_dtype pos_t,
                                   const uint32_t *q_sorted, const int32_t *cell_start,
                                   const int32_t *perm, int32_t C, const void *vals,
                                   pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                   void *mesh_vals, int32_t tile_rows, int32_t blocks, void *ws,
                                   size_t ws_bytes, void *stream)
{
    if (!plan || !pos_sorted || !q_sorted || !cell_start || !perm || !vals || !mesh_vals || !ws)
        return PFEM_ERR_INVALID_ARG;
    if (C < 1 || C > 8 || blocks < 1 || ws_bytes < 256 || nodes_total < 0) return PFEM_ERR_INVALID_ARG;
    const int sidx = tile_rows == 4 ? 0 : tile_rows == 8 ? 1 : tile_rows == 16 ? 2 : -1;
    if (sidx < 0) return PFEM_ERR_INVALID_ARG;
    if (shape != PFEM_SHAPE_LINEAR && shape != PFEM_SHAPE_QUADRATIC) return PFEM_ERR_INVALID_ARG;
    if (val_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)) return PFEM_ERR_INVALID_ARG;
    if (val_t == PFEM_F32 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    if (val_t == PFEM_BF16) return PFEM_ERR_INVALID_ARG;
    if (solve < PFEM_SOLVE_F64 || solve > PFEM_SOLVE_F32_REFINED) return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_batch_p2m(plan, pos_sorted, q_sorted, cell_start, perm, C, vals, val_t,
                                      shape, solve, mesh_vals, sidx, blocks, nodes_total, ws,
                                      ws_bytes, (cudaStream_t)stream));
}

pfem_status pfem_batch_interp_m2p(const void *plan, const void *pos, pfem_dtype pos_t, int32_t C,
                                  const void *mesh_vals, void *vals, pfem_dtype val_t,
                                  int32_t blocks, void *stream)
{
    if (!plan || !pos || !mesh_vals || !vals || C < 1 || C > 8 || blocks < 1) return PFEM_ERR_INVALID_ARG;
    if (!((val_t == PFEM_F64 && pos_t == PFEM_F64) || (val_t == PFEM_F32 && pos_t == PFEM_F32)))
        return PFEM_ERR_INVALID_ARG;
    return from_cuda(launch_batch_m2p(plan, pos, pos_t, C, mesh_vals, vals, val_t, blocks,
                                      (cudaStream_t)stream));
}

}  // extern "C"
