// capi.cu -- the extern "C" entry points declared in include/pfem.h: argument checks,
// workspace layout and dispatch to the kernels.  No entry point allocates device memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.h"

using namespace pfem;

namespace pfem {

static std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            return 152;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Binning scratch for nb*nb bins and N particles; with a mesh (n > 0) the total also covers
// what quadratic P2M keeps in the workspace once the cells are built (the queue of nodes for
// the SVD pass and the per-node records of the two-kernel path).
WsLayout ws_layout(int n, int nb, long long N, int C)
{
    (void)C;
    WsLayout L = ws_layout_bins((long long)nb * nb, N);
    if (n > 0) L.total = std::max(L.total, p2m_ws_bytes((long long)n * n, N));
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

// ----------------------------------------------------------------- contexts and errors

struct pfem_ctx {
    pfem_options opt;
    char err[512];
    void *events[8];            // stage events (cudaEvent_t) recorded by pfem_project_p2m
    int nevents;
    void *vals_event;           // event pfem_project_p2m waits on before reading the values
};

static thread_local char t_err[512];

static char *err_buf(const pfem_ctx *c) { return c ? const_cast<char *>(c->err) : t_err; }

static pfem_status say(const pfem_ctx *c, pfem_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err_buf(c), 512, fmt, ap);
    va_end(ap);
    return s;
}

static pfem_status ok(const pfem_ctx *c)
{
    err_buf(c)[0] = 0;
    return PFEM_OK;
}

static pfem_status cuda_result(const pfem_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return ok(c);
    return say(c, PFEM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void fill_defaults(pfem_options *o)
{
    if (o->walk_max_steps == 0) o->walk_max_steps = 64;
    if (o->star_capacity == 0) o->star_capacity = PFEM_KMAX;
    if (o->node_capacity == 0) o->node_capacity = PFEM_UMAX;
    if (o->batch_tile_rows == 0) o->batch_tile_rows = 8;
}

static pfem_options opts_of(const pfem_ctx *c)
{
    pfem_options o;
    if (c) o = c->opt;
    else memset(&o, 0, sizeof(o));
    fill_defaults(&o);
    return o;
}

static const char *check_options(const pfem_options &o)
{
    if (o.walk_max_steps < -1) return "walk_max_steps must be -1 (none), 0 (default) or positive";
    if (o.star_capacity != 0 && (o.star_capacity < 3 || o.star_capacity > PFEM_KMAX))
        return "star_capacity must be 0 (default) or 3..PFEM_KMAX";
    if (o.node_capacity != 0 && (o.node_capacity < 3 || o.node_capacity > PFEM_UMAX))
        return "node_capacity must be 0 (default) or 3..PFEM_UMAX";
    if (o.search_radius_max < 0) return "search_radius_max must be 0 (default) or positive";
    if (o.batch_tile_rows != 0 && o.batch_tile_rows != 4 && o.batch_tile_rows != 8 &&
        o.batch_tile_rows != 16)
        return "batch_tile_rows must be 0 (default), 4, 8 or 16";
    if (o.batch_p2m_blocks < 0 || o.batch_m2p_blocks < 0) return "block counts must be >= 0";
    for (size_t i = 0; i < sizeof(o.reserved) / sizeof(o.reserved[0]); ++i)
        if (o.reserved[i] != 0) return "reserved fields must be zero";
    return nullptr;
}

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

// Geometry arguments of one problem; a message in the context's error text when invalid.
static pfem_status make_geo(const pfem_ctx *ctx, const char *fn, int32_t n, int32_t nb,
                            int64_t N, const void *pos_sorted, pfem_dtype pos_t,
                            const uint32_t *q_sorted, const int32_t *cell_start, GeoArgs *g)
{
    if (!geom_ok(n, nb, N))
        return say(ctx, PFEM_ERR_INVALID_ARG,
                   "%s: sizes out of range (n = %d >= 9, nb = %d >= 8 with nb^2 < 2^30, 3 <= N = %lld < 2^31)",
                   fn, n, nb, (long long)N);
    if (!pos_sorted || !q_sorted || !cell_start)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: pos_sorted, q_sorted and cell_start must not be NULL", fn);
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: pos_t must be PFEM_F64 or PFEM_F32", fn);
    const pfem_options o = opts_of(ctx);
    g->n = n;
    g->nb = nb;
    g->N = N;
    g->pos_sorted = pos_sorted;
    g->pos_t = pos_t;
    g->q_sorted = q_sorted;
    g->cell_start = cell_start;
    // first search radius, largest radius, and the distance cutoff of the first star attempt
    // (2.0 mean particle spacings, fixed point: above the largest Delaunay circumdiameter of
    // jittered lattices at jitter 0.25, 1.97 spacings; a star that fails it takes the retry)
    radii_for(nb, N, &g->R0, &g->rmax, &g->dmax);
    if (g->rmax < g->R0)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: nb = %d is too small for N = %lld particles",
                   fn, nb, (long long)N);
    // the retry and fix passes search up to a quarter of the torus (regions wider than that
    // would alias in 32-bit fixed-point differences), or the context's limit
    int far = nb / 4 - 1;
    if (o.search_radius_max > 0) far = std::min(far, o.search_radius_max);
    g->rmax_far = std::max(g->rmax, far);
    g->kcap = o.star_capacity;
    g->walk_cap = o.walk_max_steps < 0 ? 0 : o.walk_max_steps;
    g->ucap = o.node_capacity;
    g->events = ctx && ctx->nevents > 0 ? ctx->events : nullptr;
    g->nevents = ctx ? ctx->nevents : 0;
    g->vals_event = ctx ? ctx->vals_event : nullptr;
    return PFEM_OK;
}

static bool solve_ok(pfem_solve s) { return s >= PFEM_SOLVE_F64 && s <= PFEM_SOLVE_F32_REFINED_FF; }
static bool shape_ok(pfem_shape s) { return s == PFEM_SHAPE_LINEAR || s == PFEM_SHAPE_QUADRATIC; }

extern "C" {

int pfem_abi_version(void) { return 2; }

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

void pfem_options_default(pfem_options *opt)
{
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    fill_defaults(opt);
}

pfem_status pfem_create(pfem_ctx **ctx, const pfem_options *opt)
{
    if (!ctx) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_create: ctx must not be NULL");
    *ctx = nullptr;
    pfem_options o;
    if (opt) o = *opt;
    else memset(&o, 0, sizeof(o));
    if (const char *why = check_options(o)) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_create: %s", why);
    pfem_ctx *c = new (std::nothrow) pfem_ctx;
    if (!c) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_create: out of host memory");
    c->opt = o;
    c->err[0] = 0;
    c->nevents = 0;
    c->vals_event = nullptr;
    *ctx = c;
    return ok(nullptr);
}

void pfem_destroy(pfem_ctx *ctx) { delete ctx; }

pfem_status pfem_get_options(const pfem_ctx *ctx, pfem_options *opt)
{
    if (!opt) return say(ctx, PFEM_ERR_INVALID_ARG, "pfem_get_options: opt must not be NULL");
    *opt = opts_of(ctx);
    return ok(ctx);
}

const char *pfem_last_error(const pfem_ctx *ctx) { return err_buf(ctx); }

pfem_status pfem_set_values_event(pfem_ctx *ctx, void *event)
{
    if (!ctx) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_set_values_event: needs a context");
    ctx->vals_event = event;
    return ok(ctx);
}

pfem_status pfem_set_stage_events(pfem_ctx *ctx, void *const *events, int32_t count)
{
    if (!ctx) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_set_stage_events: needs a context");
    if (count < 0 || count > 8 || (count > 0 && !events))
        return say(ctx, PFEM_ERR_INVALID_ARG, "pfem_set_stage_events: count must be 0..8");
    for (int i = 0; i < count; ++i) ctx->events[i] = events[i];
    ctx->nevents = count;
    return ok(ctx);
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
    if (!ws || !status_host) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_read_status: NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    DevStatus h;
    cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_result(nullptr, e, "pfem_read_status");
    *status_host = h.code;
    if (detail_host) *detail_host = h.code ? h.detail : -1;
    return PFEM_OK;
}

pfem_status pfem_get_device_status(pfem_ctx *ctx, const void *ws, int32_t *status_host,
                                   int64_t *detail_host, void *stream)
{
    if (!ws || !status_host) return say(ctx, PFEM_ERR_INVALID_ARG, "pfem_get_device_status: NULL argument");
    DevStatus h;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_result(ctx, e, "pfem_get_device_status");
    *status_host = h.code;
    if (detail_host) *detail_host = h.code ? h.detail : -1;
    if (h.code)
        return say(ctx, PFEM_OK, "device status %s (%d failures; first at index %lld)",
                   pfem_status_string((pfem_status)h.code), h.count, (long long)h.detail);
    return ok(ctx);
}

pfem_status pfem_reset_status(void *ws, void *stream)
{
    if (!ws) return say(nullptr, PFEM_ERR_INVALID_ARG, "pfem_reset_status: ws must not be NULL");
    return cuda_result(nullptr, cudaMemsetAsync(ws, 0, sizeof(DevStatus), (cudaStream_t)stream),
                       "pfem_reset_status");
}

pfem_status pfem_build_cells(pfem_ctx *ctx, int32_t nb, int64_t N, const void *pos,
                             pfem_dtype pos_t, int32_t *cell_start, int32_t *perm,
                             void *pos_sorted, uint32_t *q_sorted, void *ws, size_t ws_bytes,
                             void *stream)
{
    const char *fn = "pfem_build_cells";
    if (nb < 1 || (long long)nb * nb >= (1LL << 30) || N < 0 || N >= (1LL << 31))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: nb = %d or N = %lld out of range", fn, nb, (long long)N);
    if (!cell_start || !ws || (N > 0 && (!pos || !perm || !pos_sorted || !q_sorted)))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: pos_t must be PFEM_F64 or PFEM_F32", fn);
    const WsLayout L = ws_layout(0, nb, N, 1);
    if (ws_bytes < L.total)
        return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes = %zu < %zu", fn, ws_bytes, L.total);
    return cuda_result(ctx, launch_build_cells(nb, N, pos, pos_t, cell_start, perm, pos_sorted,
                                               q_sorted, L, ws, (cudaStream_t)stream), fn);
}

pfem_status pfem_delaunay_stars(pfem_ctx *ctx, int32_t nb, int64_t N, const uint32_t *q_sorted,
                                const int32_t *cell_start, int32_t *nbrs, int32_t *counts,
                                void *ws, size_t ws_bytes, void *stream)
{
    const char *fn = "pfem_delaunay_stars";
    GeoArgs g;
    pfem_status st = make_geo(ctx, fn, 9, nb, N, q_sorted, PFEM_F32, q_sorted, cell_start, &g);
    if (st != PFEM_OK) return st;
    if (!nbrs || !counts || !ws) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (ws_bytes < stars_ws_bytes(N))
        return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes = %zu < %zu", fn, ws_bytes, stars_ws_bytes(N));
    return cuda_result(ctx, launch_stars(g, nbrs, counts, (DevStatus *)ws, (cudaStream_t)stream), fn);
}

pfem_status pfem_shape_quadratic(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N,
                                 const void *pos_sorted, pfem_dtype pos_t,
                                 const uint32_t *q_sorted, const int32_t *cell_start,
                                 pfem_shape shape, pfem_solve solve, int32_t K, int32_t *w_idx,
                                 void *w, pfem_dtype w_t, void *ws, size_t ws_bytes, void *stream)
{
    const char *fn = "pfem_shape_quadratic";
    GeoArgs g;
    pfem_status st = make_geo(ctx, fn, n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g);
    if (st != PFEM_OK) return st;
    if (!w_idx || !w || !ws) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (K < 3 || K > PFEM_KW_MAX) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: K = %d outside 3..PFEM_KW_MAX", fn, K);
    if (!shape_ok(shape) || !solve_ok(solve)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown shape or solve", fn);
    // FP64 weights come from FP64 positions with the FP64 solve; FP32 weights from FP32 positions
    if ((w_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)) ||
        (w_t == PFEM_F32 && pos_t != PFEM_F32) || w_t == PFEM_BF16)
        return say(ctx, PFEM_ERR_INVALID_ARG,
                   "%s: FP64 weights need FP64 positions and the FP64 solve, FP32 weights FP32 positions", fn);
    if (ws_bytes < 256) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes < 256", fn);
    return cuda_result(ctx, launch_shape(g, shape, solve, K, w_idx, w, w_t, (DevStatus *)ws,
                                         ws_bytes, (cudaStream_t)stream), fn);
}

pfem_status pfem_project_p2m(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N,
                             const void *pos_sorted, pfem_dtype pos_t, const uint32_t *q_sorted,
                             const int32_t *cell_start, const int32_t *perm, int32_t C,
                             const void *vals, pfem_dtype val_t, pfem_shape shape,
                             pfem_solve solve, const int32_t *w_idx, const void *w, int32_t K,
                             pfem_dtype w_t, void *mesh_vals, void *ws, size_t ws_bytes,
                             void *stream)
{
    const char *fn = "pfem_project_p2m";
    GeoArgs g;
    pfem_status st = make_geo(ctx, fn, n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g);
    if (st != PFEM_OK) return st;
    if (C < 1 || C > 8) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: C = %d outside 1..8", fn, C);
    if (!vals || !mesh_vals || !ws) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (val_t != PFEM_F64 && val_t != PFEM_F32 && val_t != PFEM_BF16)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown val_t", fn);
    if (ws_bytes < 256) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes < 256", fn);
    cudaStream_t s = (cudaStream_t)stream;
    if (w_idx || w) {
        if (!w_idx || !w || K < 3 || K > PFEM_KW_MAX)
            return say(ctx, PFEM_ERR_INVALID_ARG, "%s: explicit weights need w_idx, w and K in 3..PFEM_KW_MAX", fn);
        if (!((val_t == PFEM_F64 && w_t == PFEM_F64) || (val_t != PFEM_F64 && w_t == PFEM_F32)))
            return say(ctx, PFEM_ERR_INVALID_ARG, "%s: weights dtype does not match the values", fn);
        cudaError_t e = wait_values(g, s);
        if (e == cudaSuccess) e = launch_apply(n, perm, C, vals, val_t, w_idx, w, K, w_t, mesh_vals, s);
        return cuda_result(ctx, e, fn);
    }
    if (!shape_ok(shape) || !solve_ok(solve)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown shape or solve", fn);
    // FP64 values use FP64 positions and the FP64 solve; FP32/BF16 values use FP32 positions
    if (val_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP64 values need FP64 positions and the FP64 solve", fn);
    if (val_t != PFEM_F64 && pos_t != PFEM_F32)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP32 and BF16 values need FP32 positions", fn);
    return cuda_result(ctx, launch_p2m(g, perm, C, vals, val_t, shape, solve, mesh_vals,
                                       (DevStatus *)ws, ws_bytes, s), fn);
}

pfem_status pfem_interp_m2p(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos,
                            pfem_dtype pos_t, int32_t C, const void *mesh_vals, void *vals,
                            pfem_dtype val_t, void *stream)
{
    const char *fn = "pfem_interp_m2p";
    if (n < 9 || N < 0 || N >= (1LL << 40) || C < 1 || C > 8)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: n = %d, N = %lld or C = %d out of range", fn, n, (long long)N, C);
    if (N > 0 && (!pos || !mesh_vals || !vals)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if ((pos_t != PFEM_F64 && pos_t != PFEM_F32) ||
        (val_t != PFEM_F64 && val_t != PFEM_F32 && val_t != PFEM_BF16))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown dtype", fn);
    return cuda_result(ctx, launch_m2p(n, N, pos, pos_t, C, mesh_vals, vals, val_t,
                                       (cudaStream_t)stream), fn);
}

size_t pfem_backward_workspace_size(int32_t n, int64_t N, int32_t K)
{
    if (n < 1 || N < 0 || K < 0) return 0;
    return bwd_layout(n, N, K).total;
}

pfem_status pfem_interp_m2p_quadratic(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos,
                                      pfem_dtype pos_t, int32_t C, const void *mesh_vals,
                                      void *vals, pfem_dtype val_t, void *stream)
{
    const char *fn = "pfem_interp_m2p_quadratic";
    if (n < 9 || N < 0 || N >= (1LL << 40) || C < 1 || C > 8)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: n = %d, N = %lld or C = %d out of range", fn, n, (long long)N, C);
    if (N > 0 && (!pos || !mesh_vals || !vals)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (!((val_t == PFEM_F64 && pos_t == PFEM_F64) || (val_t != PFEM_F64 && pos_t == PFEM_F32)))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP64 values need FP64 positions, others FP32", fn);
    return cuda_result(ctx, launch_m2p_quadratic(n, N, pos, pos_t, C, mesh_vals, vals, val_t,
                                                 (cudaStream_t)stream), fn);
}

pfem_status pfem_project_backward(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N,
                                  const void *pos_sorted, pfem_dtype pos_t,
                                  const uint32_t *q_sorted, const int32_t *cell_start,
                                  const int32_t *perm, int32_t C, const void *vals,
                                  pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                  pfem_backward_mode mode, const int32_t *w_idx, const void *w,
                                  int32_t K, pfem_dtype w_t, const void *grad_mesh,
                                  void *grad_vals, void *grad_pos, void *ws, size_t ws_bytes,
                                  void *stream)
{
    const char *fn = "pfem_project_backward";
    GeoArgs g;
    pfem_status st = make_geo(ctx, fn, n, nb, N, pos_sorted, pos_t, q_sorted, cell_start, &g);
    if (st != PFEM_OK) return st;
    if (C < 1 || C > 8) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: C = %d outside 1..8", fn, C);
    if (!vals || !grad_mesh || !grad_vals || !ws) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (!shape_ok(shape)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown shape", fn);
    if (val_t == PFEM_F64) {
        if (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)
            return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP64 values need FP64 positions and the FP64 solve", fn);
    } else if (val_t == PFEM_F32) {
        if (pos_t != PFEM_F32 || (solve != PFEM_SOLVE_F64 && solve != PFEM_SOLVE_F32))
            return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP32 values need FP32 positions and the FP64 or FP32 solve", fn);
    } else {
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: values must be FP64 or FP32", fn);
    }
    const bool ckpt = mode == PFEM_BACKWARD_CHECKPOINT;
    if (mode != PFEM_BACKWARD_RECOMPUTE && !ckpt) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown mode", fn);
    if (ckpt && (!w_idx || !w || K < 3 || K > PFEM_KW_MAX || w_t != val_t))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: checkpoint mode needs w_idx, w (dtype of the values) and K in 3..PFEM_KW_MAX", fn);
    const BwdLayout L = bwd_layout(n, N, ckpt ? K : 0);
    if (ws_bytes < L.total) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes = %zu < %zu", fn, ws_bytes, L.total);
    return cuda_result(ctx, launch_p2m_backward(g, perm, C, vals, val_t, shape, solve, ckpt, w_idx,
                                                w, ckpt ? K : 0, grad_mesh, grad_vals, grad_pos, L,
                                                ws, (cudaStream_t)stream), fn);
}

pfem_status pfem_interp_m2p_backward(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N,
                                     const void *pos, pfem_dtype pos_t, const int32_t *cell_start,
                                     const int32_t *perm, int32_t C, const void *mesh_vals,
                                     const void *grad_vals, pfem_dtype val_t, void *grad_mesh,
                                     void *grad_pos, void *stream)
{
    const char *fn = "pfem_interp_m2p_backward";
    if (n < 9 || nb < 1 || (long long)nb * nb >= (1LL << 30) || N < 0 || N >= (1LL << 31) ||
        C < 1 || C > 8)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: sizes out of range", fn);
    if (!cell_start || !grad_mesh || (N > 0 && (!pos || !perm || !grad_vals)) ||
        (grad_pos && !mesh_vals))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if ((pos_t != PFEM_F64 && pos_t != PFEM_F32) || (val_t != PFEM_F64 && val_t != PFEM_F32))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown dtype", fn);
    return cuda_result(ctx, launch_m2p_backward(n, nb, N, pos, pos_t, cell_start, perm, C,
                                                mesh_vals, grad_vals, val_t, grad_mesh, grad_pos,
                                                (cudaStream_t)stream), fn);
}

pfem_status pfem_advect_midpoint(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos,
                                 pfem_dtype pos_t, const void *mesh_vel, double dt, void *pos_out,
                                 void *stream)
{
    const char *fn = "pfem_advect_midpoint";
    if (n < 9 || N < 0 || N >= (1LL << 40)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: n or N out of range", fn);
    if (N > 0 && (!pos || !mesh_vel || !pos_out)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown pos_t", fn);
    if (!(std::fabs(dt) < 1e30)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: dt is not finite", fn);
    if (N == 0) return ok(ctx);
    return cuda_result(ctx, launch_advect_midpoint(n, N, pos, pos_t, mesh_vel, dt, pos_out,
                                                   (cudaStream_t)stream), fn);
}

size_t pfem_update_workspace_size(int32_t nb, int64_t N)
{
    if (nb < 1 || N < 0) return 0;
    return update_ws_bytes((long long)nb * nb, N);
}

pfem_status pfem_update_cells(pfem_ctx *ctx, int32_t nb, int64_t N, const void *pos,
                              pfem_dtype pos_t, const int32_t *cell_start_old,
                              const int32_t *perm_old, const uint32_t *q_sorted_old,
                              int32_t *cell_start, int32_t *perm, void *pos_sorted,
                              uint32_t *q_sorted, void *ws, size_t ws_bytes, void *stream)
{
    const char *fn = "pfem_update_cells";
    if (nb < 3 || (long long)nb * nb >= (1LL << 30) || N < 0 || N >= (1LL << 31))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: nb = %d (>= 3) or N = %lld out of range", fn, nb, (long long)N);
    if (!cell_start_old || !cell_start || !ws ||
        (N > 0 && (!pos || !perm_old || !q_sorted_old || !perm || !pos_sorted || !q_sorted)))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (cell_start == cell_start_old || perm == perm_old || q_sorted == q_sorted_old)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: the new arrays must not alias the old ones", fn);
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown pos_t", fn);
    const size_t need = update_ws_bytes((long long)nb * nb, N);
    if (ws_bytes < need) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes = %zu < %zu", fn, ws_bytes, need);
    return cuda_result(ctx, launch_update_cells(nb, N, pos, pos_t, cell_start_old, perm_old,
                                                q_sorted_old, cell_start, perm, pos_sorted,
                                                q_sorted, ws, (cudaStream_t)stream), fn);
}

size_t pfem_batch_plan_size(int32_t P)
{
    return P < 1 ? 0 : batch_plan_bytes(P);
}

pfem_status pfem_batch_plan_init(pfem_ctx *ctx, int32_t P, const pfem_batch_problem *problems,
                                 void *plan, int64_t *totals)
{
    const char *fn = "pfem_batch_plan_init";
    if (P < 1 || !problems || !plan || !totals) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: bad argument", fn);
    long long Nt = 0, bt = 0, nt = 0;
    const int st = batch_plan_build(P, problems, plan, &Nt, &bt, &nt);
    if (st == PFEM_ERR_CUDA) return say(ctx, PFEM_ERR_CUDA, "%s: copying the plan failed", fn);
    if (st != PFEM_OK)
        return say(ctx, (pfem_status)st, "%s: a problem's sizes are out of range (n >= 9, nb >= 8, N >= 3, totals < 2^31)", fn);
    totals[0] = Nt;
    totals[1] = bt;
    totals[2] = nt;
    return ok(ctx);
}

size_t pfem_batch_workspace_size(int64_t N_total, int64_t bins_total, int64_t nodes_total)
{
    if (N_total < 0 || bins_total < 1 || nodes_total < 0) return 0;
    const size_t b = ws_layout_bins(bins_total, N_total).total;
    return nodes_total > 0 ? std::max(b, batch_p2m_ws_bytes(nodes_total, N_total)) : b;
}

pfem_status pfem_batch_build_cells(pfem_ctx *ctx, const void *plan, int64_t N_total,
                                   int64_t bins_total, const void *pos, pfem_dtype pos_t,
                                   int32_t *cell_start, int32_t *perm, void *pos_sorted,
                                   uint32_t *q_sorted, void *ws, size_t ws_bytes, void *stream)
{
    const char *fn = "pfem_batch_build_cells";
    if (!plan || !pos || !cell_start || !perm || !pos_sorted || !q_sorted || !ws)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (N_total < 1 || N_total >= (1LL << 31) || bins_total < 1 || bins_total >= (1LL << 31))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: totals out of range", fn);
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown pos_t", fn);
    const WsLayout L = ws_layout_bins(bins_total, N_total);
    if (ws_bytes < L.total) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes = %zu < %zu", fn, ws_bytes, L.total);
    return cuda_result(ctx, launch_batch_build_cells(plan, N_total, bins_total, pos, pos_t,
                                                     cell_start, perm, pos_sorted, q_sorted, L,
                                                     ws, (cudaStream_t)stream), fn);
}

pfem_status pfem_batch_project_p2m(pfem_ctx *ctx, const void *plan, int64_t nodes_total,
                                   int64_t N_total, const void *pos_sorted, pfem_dtype pos_t,
                                   const uint32_t *q_sorted, const int32_t *cell_start,
                                   const int32_t *perm, int32_t C, const void *vals,
                                   pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                   void *mesh_vals, int32_t tile_rows, int32_t blocks, void *ws,
                                   size_t ws_bytes, void *stream)
{
    const char *fn = "pfem_batch_project_p2m";
    const pfem_options o = opts_of(ctx);
    if (!plan || !pos_sorted || !q_sorted || !cell_start || !perm || !vals || !mesh_vals || !ws)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: NULL buffer", fn);
    if (tile_rows == 0) tile_rows = o.batch_tile_rows;
    if (blocks == 0) blocks = o.batch_p2m_blocks > 0 ? o.batch_p2m_blocks : num_sms() * 8;
    if (C < 1 || C > 8 || blocks < 1 || nodes_total < 0 || N_total < 0)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: C, blocks or totals out of range", fn);
    if (ws_bytes < 256) return say(ctx, PFEM_ERR_WORKSPACE, "%s: ws_bytes < 256", fn);
    const int sidx = tile_rows == 4 ? 0 : tile_rows == 8 ? 1 : tile_rows == 16 ? 2 : -1;
    if (sidx < 0) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: tile_rows must be 4, 8 or 16", fn);
    if (!shape_ok(shape) || !solve_ok(solve)) return say(ctx, PFEM_ERR_INVALID_ARG, "%s: unknown shape or solve", fn);
    if ((val_t == PFEM_F64 && (pos_t != PFEM_F64 || solve != PFEM_SOLVE_F64)) ||
        (val_t == PFEM_F32 && pos_t != PFEM_F32) || val_t == PFEM_BF16)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP64 values need FP64 positions and the FP64 solve, FP32 values FP32 positions", fn);
    return cuda_result(ctx, launch_batch_p2m(plan, pos_sorted, q_sorted, cell_start, perm, C, vals,
                                             val_t, shape, solve, mesh_vals, sidx, blocks,
                                             nodes_total, N_total, ws, ws_bytes,
                                             (cudaStream_t)stream), fn);
}

pfem_status pfem_batch_interp_m2p(pfem_ctx *ctx, const void *plan, const void *pos,
                                  pfem_dtype pos_t, int32_t C, const void *mesh_vals, void *vals,
                                  pfem_dtype val_t, int32_t blocks, void *stream)
{
    const char *fn = "pfem_batch_interp_m2p";
    const pfem_options o = opts_of(ctx);
    if (blocks == 0) blocks = o.batch_m2p_blocks > 0 ? o.batch_m2p_blocks : num_sms() * 16;
    if (!plan || !pos || !mesh_vals || !vals || C < 1 || C > 8 || blocks < 1)
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: bad argument", fn);
    if (!((val_t == PFEM_F64 && pos_t == PFEM_F64) || (val_t == PFEM_F32 && pos_t == PFEM_F32)))
        return say(ctx, PFEM_ERR_INVALID_ARG, "%s: FP64 or FP32 values with positions of the same dtype", fn);
    return cuda_result(ctx, launch_batch_m2p(plan, pos, pos_t, C, mesh_vals, vals, val_t, blocks,
                                             (cudaStream_t)stream), fn);
}

}  // extern "C"
