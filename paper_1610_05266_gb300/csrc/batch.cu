// batch.cu -- many independent, uneven projection problems in one launch per stage.
//
// The batch is laid out as one concatenated problem: particles of problem p occupy
// [poff_p, poff_p + N_p) of the particle arrays, its nb_p^2 bins occupy [boff_p, ...) of one
// bin array, and its n_p^2 nodes occupy [noff_p, ...) of the mesh array.  Binning every
// particle into its problem's bins at offset boff_p turns the whole batch into a single
// stable counting sort (the same scan / scatter / per-bin sort / gather kernels as for one
// problem); slots and bin starts are then global indices, valid for every problem at once.
//
// P2M runs as a persistent kernel: a grid of (SMs x blocks per SM) blocks pulls work items
// (problem, tile of 16 x TY nodes) from an atomic counter until the batch is done.  Items
// are independent and every node is computed by the same deterministic code, so the result
// does not depend on the schedule.  M2P and the binning walk fixed-size particle chunks.
// A plan (descriptors and prefix tables) is built once on the host and copied to the device;
// the stage launches allocate nothing and can be captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "p2m.cuh"

namespace pfem {

struct BDesc {
    int n, nb, R0, rmax;
    float dmax;
    int pad;
    long long N, poff, boff, noff;
};

constexpr int BT_SHAPES = 3;          // node tiles 16x4, 16x8, 16x16 (64, 128, 256 threads)
constexpr int BCHUNK = 4096;          // particles per chunk

constexpr int BSTAR = 128;           // particles per block of the star-table kernel

struct BPlanDev {
    int P;
    int pad;
    long long n_items[BT_SHAPES];
    long long n_chunks;
    long long total_bins;
    long long total_particles, total_nodes;
    long long n_star_tiles;
    // followed in memory by: BDesc desc[P]; long long tile_prefix[BT_SHAPES][P+1];
    // long long chunk_prefix[P+1]; long long star_tile_prefix[P+1]
};

__host__ __device__ inline size_t plan_bytes(int P)
{
    return sizeof(BPlanDev) + sizeof(BDesc) * (size_t)P +
           sizeof(long long) * (size_t)(BT_SHAPES + 2) * (size_t)(P + 1);
}
__device__ __forceinline__ const BDesc *plan_desc(const BPlanDev *pl)
{
    return reinterpret_cast<const BDesc *>(pl + 1);
}
__device__ __forceinline__ const long long *plan_tiles(const BPlanDev *pl, int shape)
{
    return reinterpret_cast<const long long *>(plan_desc(pl) + pl->P) + (long long)shape * (pl->P + 1);
}
__device__ __forceinline__ const long long *plan_chunks(const BPlanDev *pl)
{
    return reinterpret_cast<const long long *>(plan_desc(pl) + pl->P) + (long long)BT_SHAPES * (pl->P + 1);
}
__device__ __forceinline__ const long long *plan_star_tiles(const BPlanDev *pl)
{
    return plan_chunks(pl) + (pl->P + 1);
}

// Problem of batch-wide index x, given the per-problem offsets off(p) (increasing).
template <typename F>
__device__ __forceinline__ int find_problem(int P, long long x, F &&off)
{
    int lo = 0, hi = P;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off(mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Bins and search radii of problem d within the batch's concatenated arrays.
__device__ __forceinline__ void problem_args(P2MArgs &a, const P2MArgs &base, const BDesc &d)
{
    a = base;
    a.n = d.n;
    a.B.start = base.B.start + d.boff;
    a.B.nb = d.nb;
    a.B.rmax = d.rmax;
    a.B.dmax = d.dmax;
    a.R0 = d.R0;
    a.noff = d.noff;
}

template <typename V>
__device__ __forceinline__ void problem_out(P2MArgs &a, const P2MArgs &base, const BDesc &d)
{
    a.out = base.out ? (void *)((V *)base.out + d.noff * base.C) : nullptr;
}

// index p with prefix[p] <= x < prefix[p+1]
__device__ __forceinline__ int find_item(const long long *prefix, int P, long long x)
{
    int lo = 0, hi = P;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- binning

template <typename P>
__global__ void __launch_bounds__(256) k_bin_batch(const BPlanDev *pl, const P *__restrict__ pos,
                                                   int *__restrict__ key, int *__restrict__ rank,
                                                   int *__restrict__ count)
{
    const long long *cp = plan_chunks(pl);
    for (long long c = blockIdx.x; c < pl->n_chunks; c += gridDim.x) {
        const int p = find_item(cp, pl->P, c);
        const BDesc d = plan_desc(pl)[p];
        const long long first = (c - cp[p]) * BCHUNK;
        const long long end = min(d.N, first + BCHUNK);
        for (long long i = first + threadIdx.x; i < end; i += blockDim.x) {
            const long long m = d.poff + i;
            P x, y;
            load_pos(pos, m, x, y);
            const int b = (int)(d.boff + (long long)bin_of(fx_of(y), d.nb) * d.nb + bin_of(fx_of(x), d.nb));
            key[m] = b;
            rank[m] = atomicAdd(count + b, 1);
        }
    }
}

// ---------------------------------------------------------------- P2M

// The plan and the caller's totals must agree before any record or table entry is written.
__device__ __forceinline__ bool totals_ok(const BPlanDev *pl, const NodeRecs *r, const StarTab *t,
                                          DevStatus *st)
{
    const bool ok = (!r || r->nodes == pl->total_nodes) && (!t || t->N == pl->total_particles);
    if (!ok && blockIdx.x == 0 && threadIdx.x == 0) record_error(st, PFEM_ERR_INVALID_ARG, -1);
    return ok;
}

// Per-node fused P2M (linear shape functions, or no room for the table) in a persistent loop.
template <typename P, typename V, typename R, typename S, int REFINE, int SHAPE>
__global__ void __launch_bounds__(256, PFEM_P2M_MIN_BLOCKS / 2) k_p2m_batch(const BPlanDev *pl, int shape_idx, P2MArgs base,
                            unsigned long long *counter)
{
    __shared__ long long item;
    const int TY = blockDim.x / 16;
    const long long total = pl->n_items[shape_idx];
    const long long *tp = plan_tiles(pl, shape_idx);
    for (int guard = 0; guard < (1 << 30); ++guard) {
        __syncthreads();
        if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = item;
        if (it >= total) break;
        const int p = find_item(tp, pl->P, it);
        const BDesc d = plan_desc(pl)[p];
        const long long t = it - tp[p];
        const int tiles_x = (d.n + 15) / 16;
        const int I = (int)(t % tiles_x) * 16 + (threadIdx.x & 15);
        const int J = (int)(t / tiles_x) * TY + (threadIdx.x >> 4);
        if (I >= d.n || J >= d.n) continue;
        P2MArgs a;
        problem_args(a, base, d);
        problem_out<V>(a, base, d);
        p2m_node<P, V, R, S, REFINE, SHAPE, false>(a, I, J);
    }
}

// Star table of every problem: block b takes 128 consecutive particles of one problem.
__global__ void __launch_bounds__(BSTAR) k_star_list_batch(const BPlanDev *pl, P2MArgs base,
                                                           StarTab t)
{
    __shared__ float2 sxy[STAR_KL * BSTAR];
    __shared__ unsigned skey[STAR_KL * BSTAR];
    __shared__ int ss[STAR_KL * BSTAR];
    __shared__ unsigned char sord[STAR_KL * BSTAR];
    __shared__ unsigned char sstk[STAR_KL * BSTAR];
    if (!totals_ok(pl, nullptr, &t, base.status)) return;
    const long long *sp = plan_star_tiles(pl);
    for (long long b = blockIdx.x; b < pl->n_star_tiles; b += gridDim.x) {
        const int p = find_item(sp, pl->P, b);
        const BDesc d = plan_desc(pl)[p];
        const long long i = (b - sp[p]) * BSTAR + threadIdx.x;
        if (i >= d.N) continue;
        P2MArgs a;
        problem_args(a, base, d);
        const HullList L{sxy + threadIdx.x, skey + threadIdx.x, ss + threadIdx.x, sord + threadIdx.x,
                      sstk + threadIdx.x, BSTAR};
        star_list_slot(a.B, a.R0, t, d.poff + i, L, a.status);
    }
}

// The queued particles of the table, each with its problem's bins and the widest radius: the
// hull attempt for a short queue, then the region search for the stars still queued.
template <bool HULL>
__global__ void __launch_bounds__(64) k_star_retry_batch(const BPlanDev *pl, P2MArgs base, StarTab t)
{
    __shared__ float2 sxy[HULL ? STAR_KL_RETRY * 64 : 1];
    __shared__ unsigned skey[HULL ? STAR_KL_RETRY * 64 : 1];
    __shared__ int ss[HULL ? STAR_KL_RETRY * 64 : 1];
    __shared__ unsigned char sord[HULL ? STAR_KL_RETRY * 64 : 1];
    __shared__ unsigned char sstk[HULL ? STAR_KL_RETRY * 64 : 1];
    const int n = min(*t.qcount, (int)min(t.N, (long long)0x7fffffff));
    if (HULL && !short_queue(n, t.N)) return;
    const BDesc *D = plan_desc(pl);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int v = t.queue[i];
        const int p = find_problem(pl->P, v, [&](int k) { return D[k].poff; });
        const BDesc d = D[p];
        P2MArgs a;
        problem_args(a, base, d);
        a.B.rmax = max(d.rmax, d.nb / 4 - 1);
        if constexpr (HULL) {
            const HullList L{sxy + threadIdx.x, skey + threadIdx.x, ss + threadIdx.x,
                             sord + threadIdx.x, sstk + threadIdx.x, 64};
            star_retry_hull_slot(a.B, a.R0, t, v, L, a.status);
        } else {
            star_retry_slot(a.B, a.R0, t, v, a.status);
        }
    }
}

// Node records of every problem in a persistent loop (the geometry half of the two-kernel
// quadratic P2M): each node's record at its batch-wide index, with its coordinates.
template <typename P, typename V, typename R>
__global__ void __launch_bounds__(256, PFEM_GEOM_MIN_BLOCKS / 2) k_p2m_batch_geom(
    const BPlanDev *pl, int shape_idx, P2MArgs base, unsigned long long *counter, StarTab tab,
    NodeRecs r)
{
    __shared__ long long item;
    if (!totals_ok(pl, &r, &tab, base.status)) return;
    const int TY = blockDim.x / 16;
    const long long total = pl->n_items[shape_idx];
    const long long *tp = plan_tiles(pl, shape_idx);
    for (int guard = 0; guard < (1 << 30); ++guard) {
        __syncthreads();
        if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = item;
        if (it >= total) break;
        const int p = find_item(tp, pl->P, it);
        const BDesc d = plan_desc(pl)[p];
        const long long t = it - tp[p];
        const int tiles_x = (d.n + 15) / 16;
        const int I = (int)(t % tiles_x) * 16 + (threadIdx.x & 15);
        const int J = (int)(t / tiles_x) * TY + (threadIdx.x >> 4);
        if (I >= d.n || J >= d.n) continue;
        const long long rec = d.noff + (long long)J * d.n + I;
        if (rec >= r.nodes) continue;
        P2MArgs a;
        problem_args(a, base, d);
        problem_out<V>(a, base, d);
        geom_node<P, V, R>(a, tab, r, I, J, rec);
    }
}

// The table path's fast pass of every problem in one persistent kernel (as k_p2m_tab: location
// from the star table, edge solves and apply per node, no node records).
template <typename P, typename V, typename R, typename S, int REFINE>
__global__ void __launch_bounds__(256, tab_min_blocks<S, REFINE>() / 2) k_p2m_batch_tab(
    const BPlanDev *pl, int shape_idx, P2MArgs base, unsigned long long *counter, StarTab tab)
{
    __shared__ long long item;
    if (!totals_ok(pl, nullptr, &tab, base.status)) return;
    const int TY = blockDim.x / 16;
    const long long total = pl->n_items[shape_idx];
    const long long *tp = plan_tiles(pl, shape_idx);
    for (int guard = 0; guard < (1 << 30); ++guard) {
        __syncthreads();
        if (threadIdx.x == 0) item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long it = item;
        if (it >= total) break;
        const int p = find_item(tp, pl->P, it);
        const BDesc d = plan_desc(pl)[p];
        const long long t = it - tp[p];
        const int tiles_x = (d.n + 15) / 16;
        const int I = (int)(t % tiles_x) * 16 + (threadIdx.x & 15);
        const int J = (int)(t / tiles_x) * TY + (threadIdx.x >> 4);
        if (I >= d.n || J >= d.n) continue;
        P2MArgs a;
        problem_args(a, base, d);
        problem_out<V>(a, base, d);
        tab_node<P, V, R, S, REFINE>(a, tab, I, J);
    }
}

// The fix pass over the batch's queued nodes (batch-wide indices), each with its problem's
// bins, the widest search radius and FP64 SVD solves.
template <typename P, typename V, typename R, int SHAPE>
__global__ void __launch_bounds__(128) k_p2m_fix_batch(const BPlanDev *pl, P2MArgs base)
{
    const int cnt = min(*base.defer_count, base.defer_cap);
    const BDesc *D = plan_desc(pl);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const long long g = base.defer_list[i];
        const int p = find_problem(pl->P, g, [&](int k) { return D[k].noff; });
        const BDesc d = D[p];
        P2MArgs a;
        problem_args(a, base, d);
        problem_out<V>(a, base, d);
        a.defer_cap = 0;
        a.B.rmax = max(d.rmax, d.nb / 4 - 1);
        const long long node = g - d.noff;
        p2m_node<P, V, R, double, REFINE_NONE, SHAPE, false, true>(a, (int)(node % d.n),
                                                                  (int)(node / d.n));
    }
}

// ---------------------------------------------------------------- M2P

template <typename P, typename V, typename R>
__global__ void __launch_bounds__(256) k_m2p_batch(const BPlanDev *pl, const P *__restrict__ pos,
                                                   int C, const V *__restrict__ mesh,
                                                   V *__restrict__ vals)
{
    const long long *cp = plan_chunks(pl);
    for (long long c = blockIdx.x; c < pl->n_chunks; c += gridDim.x) {
        const int p = find_item(cp, pl->P, c);
        const BDesc d = plan_desc(pl)[p];
        const int n = d.n, nc = n - 1;
        const V *mp = mesh + d.noff * C;
        const long long first = (c - cp[p]) * BCHUNK;
        const long long end = min(d.N, first + BCHUNK);
        for (long long i = first + threadIdx.x; i < end; i += blockDim.x) {
            const long long m = d.poff + i;
            P px, py;
            load_pos(pos, m, px, py);
            const int ci = bin_of(fx_of(px), nc), cj = bin_of(fx_of(py), nc);
            P s = fma(px - floor(px), (P)nc, (P)(-ci)), t = fma(py - floor(py), (P)nc, (P)(-cj));
            if (s > (P)(0.5 * nc)) s -= (P)nc;
            if (t > (P)(0.5 * nc)) t -= (P)nc;
            const long long n00 = (long long)cj * n + ci;
            long long nb_, nc_;
            R w0, w1, w2;
            if (s >= t) { nb_ = n00 + 1; nc_ = n00 + n + 1; w0 = R(P(1) - s); w1 = R(s - t); w2 = R(t); }
            else        { nb_ = n00 + n + 1; nc_ = n00 + n; w0 = R(P(1) - t); w1 = R(s); w2 = R(t - s); }
            for (int k = 0; k < C; ++k) {
                const R v = w0 * load_val<V, R>(mp + n00 * C + k) + w1 * load_val<V, R>(mp + nb_ * C + k) +
                            w2 * load_val<V, R>(mp + nc_ * C + k);
                store_val<V, R>(vals + m * C + k, v);
            }
        }
    }
}

// ---------------------------------------------------------------- host side

size_t batch_plan_bytes(int P) { return plan_bytes(P); }

void radii_for(int nb, long long N, int *R0, int *rmax, float *dmax);

int batch_plan_build(int P, const pfem_batch_problem *probs, void *plan_dev, long long *N_total,
                     long long *bins_total, long long *nodes_total)
{
    std::vector<unsigned char> buf(plan_bytes(P));
    BPlanDev *pl = reinterpret_cast<BPlanDev *>(buf.data());
    BDesc *desc = reinterpret_cast<BDesc *>(pl + 1);
    long long *tiles = reinterpret_cast<long long *>(desc + P);
    long long *chunks = tiles + (long long)BT_SHAPES * (P + 1);
    long long *stiles = chunks + (P + 1);
    pl->P = P;
    long long poff = 0, boff = 0, noff = 0;
    const int TYs[BT_SHAPES] = {4, 8, 16};
    for (int s = 0; s < BT_SHAPES; ++s) tiles[(long long)s * (P + 1)] = 0;
    chunks[0] = 0;
    stiles[0] = 0;
    for (int p = 0; p < P; ++p) {
        const pfem_batch_problem &q = probs[p];
        if (q.n < 9 || q.nb < 8 || q.N < 3 || (long long)q.nb * q.nb >= (1LL << 30)) return PFEM_ERR_INVALID_ARG;
        BDesc &d = desc[p];
        d.n = q.n;
        d.nb = q.nb;
        d.N = q.N;
        radii_for(q.nb, q.N, &d.R0, &d.rmax, &d.dmax);
        if (d.rmax < d.R0) return PFEM_ERR_INVALID_ARG;
        d.pad = 0;
        d.poff = poff;
        d.boff = boff;
        d.noff = noff;
        poff += q.N;
        boff += (long long)q.nb * q.nb;
        noff += (long long)q.n * q.n;
        for (int s = 0; s < BT_SHAPES; ++s) {
            const long long tl = (long long)((q.n + 15) / 16) * ((q.n + TYs[s] - 1) / TYs[s]);
            tiles[(long long)s * (P + 1) + p + 1] = tiles[(long long)s * (P + 1) + p] + tl;
        }
        chunks[p + 1] = chunks[p] + (q.N + BCHUNK - 1) / BCHUNK;
        stiles[p + 1] = stiles[p] + (q.N + BSTAR - 1) / BSTAR;
    }
    if (poff >= (1LL << 31) || boff >= (1LL << 31)) return PFEM_ERR_INVALID_ARG;
    for (int s = 0; s < BT_SHAPES; ++s) pl->n_items[s] = tiles[(long long)s * (P + 1) + P];
    pl->n_chunks = chunks[P];
    pl->n_star_tiles = stiles[P];
    pl->total_bins = boff;
    pl->total_particles = poff;
    pl->total_nodes = noff;
    *N_total = poff;
    *bins_total = boff;
    *nodes_total = noff;
    if (cudaMemcpy(plan_dev, buf.data(), buf.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return PFEM_ERR_CUDA;
    return PFEM_OK;
}

cudaError_t launch_batch_build_cells(const void *plan, long long Ntot, long long bins_total,
                                     const void *pos, pfem_dtype pos_t, int *cell_start, int *perm,
                                     void *pos_sorted, uint32_t *q_sorted, const WsLayout &L,
                                     void *ws, cudaStream_t s)
{
    char *W = (char *)ws;
    int *count = (int *)(W + L.count), *key = (int *)(W + L.key), *rank = (int *)(W + L.rank);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(bins_total + 1), s);
    if (e != cudaSuccess) return e;
    const BPlanDev *pl = (const BPlanDev *)plan;
    if (pos_t == PFEM_F64)
        k_bin_batch<double><<<num_sms() * 8, 256, 0, s>>>(pl, (const double *)pos, key, rank, count);
    else
        k_bin_batch<float><<<num_sms() * 8, 256, 0, s>>>(pl, (const float *)pos, key, rank, count);
    count_launch();
    e = scan_exclusive(count, cell_start, bins_total + 1, (int *)(W + L.scan), s);
    if (e != cudaSuccess) return e;
    return launch_sort_gather(bins_total, Ntot, pos, pos_t, key, rank, cell_start, perm, pos_sorted,
                              q_sorted, s);
}

// Workspace of the batched P2M: status (byte 0), work counter (byte 64), fix-pass queue counter
// (byte 128), star-table queue counter (byte 132); the fix-pass queue from byte 256 (8 bytes per
// node), then the node records (with the nodes' coordinates) and the star table.
static size_t al256b(size_t x) { return (x + 255) & ~(size_t)255; }

size_t batch_p2m_ws_bytes(long long nodes_total, long long N_total)
{
    NodeRecs r;
    return al256b(256 + 8 * (size_t)nodes_total) +
           al256b(node_recs_layout(nullptr, nodes_total, &r, true)) + star_tab_bytes(N_total);
}

struct BatchWs {
    NodeRecs recs;
    StarTab tab;
    bool table;
};

template <typename P, typename V, typename R, typename S, int REF, int SHAPE>
static cudaError_t p2m_batch_t(const void *plan, const P2MArgs &base, int shape_idx, int blocks,
                               unsigned long long *counter, const BatchWs &w, cudaStream_t s)
{
    const BPlanDev *pl = (const BPlanDev *)plan;
    // work counter, fix-pass counter and star-table counter in one clear
    cudaError_t e = cudaMemsetAsync(counter, 0, 128, s);
    if (e != cudaSuccess) return e;
    const int TYs[BT_SHAPES] = {4, 8, 16};
    if (SHAPE == PFEM_SHAPE_QUADRATIC && w.table) {
        k_star_list_batch<<<num_sms() * 8, BSTAR, 0, s>>>(pl, base, w.tab);
        k_star_retry_batch<true><<<num_sms() * PFEM_RETRY_BLOCKS, 64, 0, s>>>(pl, base, w.tab);
        k_star_retry_batch<false><<<num_sms() * PFEM_RETRY_REGION_BLOCKS, 64, 0, s>>>(pl, base, w.tab);
        if (REF != REFINE_FF) {      // one kernel, as the single-problem table path
            k_p2m_batch_tab<P, V, R, S, REF><<<blocks, 16 * TYs[shape_idx], 0, s>>>(
                pl, shape_idx, base, counter, w.tab);
            count_launch(4);
        } else {
            k_p2m_batch_geom<P, V, R><<<blocks, 16 * TYs[shape_idx], 0, s>>>(pl, shape_idx, base,
                                                                          counter, w.tab, w.recs);
            k_p2m_solve<P, V, R, S, REF><<<(unsigned)((w.recs.nodes + 127) / 128), 128, 0, s>>>(base, w.recs);
            count_launch(5);
        }
    } else {
        k_p2m_batch<P, V, R, S, REF, SHAPE><<<blocks, 16 * TYs[shape_idx], 0, s>>>(
            pl, shape_idx, base, counter);
        count_launch();
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || base.defer_cap <= 0) return e;
    k_p2m_fix_batch<P, V, R, SHAPE><<<num_sms(), 128, 0, s>>>(pl, base);
    count_launch();
    return cudaGetLastError();
}

template <typename P, typename V, int SHAPE>
static cudaError_t p2m_batch_solve(pfem_solve solve, const void *plan, const P2MArgs &a,
                                   int shape_idx, int blocks, unsigned long long *counter,
                                   const BatchWs &w, cudaStream_t s)
{
    switch (solve) {
    case PFEM_SOLVE_F64: return p2m_batch_t<P, V, float, double, REFINE_NONE, SHAPE>(plan, a, shape_idx, blocks, counter, w, s);
    case PFEM_SOLVE_F32: return p2m_batch_t<P, V, float, float, REFINE_NONE, SHAPE>(plan, a, shape_idx, blocks, counter, w, s);
    case PFEM_SOLVE_F32_REFINED: return p2m_batch_t<P, V, float, float, REFINE_F64, SHAPE>(plan, a, shape_idx, blocks, counter, w, s);
    default: return p2m_batch_t<P, V, float, float, REFINE_FF, SHAPE>(plan, a, shape_idx, blocks, counter, w, s);
    }
}

cudaError_t launch_batch_p2m(const void *plan, const void *pos_sorted, const uint32_t *q_sorted,
                             const int *cell_start, const int *perm, int C, const void *vals,
                             pfem_dtype val_t, pfem_shape shape, pfem_solve solve, void *mesh,
                             int shape_idx, int blocks, long long nodes_total, long long N_total,
                             void *ws, size_t ws_bytes, cudaStream_t s)
{
    char *W = (char *)ws;
    BatchWs w;
    w.table = nodes_total > 0 && N_total > 0 && ws_bytes >= batch_p2m_ws_bytes(nodes_total, N_total);
    P2MArgs a;
    a.n = 0;
    a.B.q = (const uint2 *)q_sorted;
    a.B.start = cell_start;
    a.B.nb = 0;
    a.B.rmax = 0;
    a.B.dmax = 0.f;
    a.R0 = 1;
    a.pos = pos_sorted;
    a.perm = perm;
    a.vals = vals;
    a.C = C;
    a.out = mesh;
    a.w_idx = nullptr;
    a.w = nullptr;
    a.K = 0;
    a.status = (DevStatus *)ws;
    // the fix-pass queue: one entry per node of the batch when the workspace holds it
    const long long qcap = nodes_total > 0 && ws_bytes >= 256 + 8 * (size_t)nodes_total ? nodes_total : 0;
    a.defer_cap = (int)std::min(qcap, (long long)0x7fffffff);
    a.defer_count = a.defer_cap > 0 ? (int *)(W + 128) : nullptr;
    a.defer_list = a.defer_cap > 0 ? (long long *)(W + 256) : nullptr;
    if (w.table) {
        char *base = W + al256b(256 + 8 * (size_t)nodes_total);
        const size_t rb = al256b(node_recs_layout(base, nodes_total, &w.recs, true));
        w.tab = star_tab_layout(base + rb, N_total, (int *)(W + 132));
    }
    unsigned long long *counter = (unsigned long long *)(W + 64);
    const bool q = shape == PFEM_SHAPE_QUADRATIC;
    if (val_t == PFEM_F64) {
        if (!q) return p2m_batch_t<double, double, double, double, REFINE_NONE, 0>(plan, a, shape_idx, blocks, counter, w, s);
        return p2m_batch_t<double, double, double, double, REFINE_NONE, 1>(plan, a, shape_idx, blocks, counter, w, s);
    }
    if (val_t == PFEM_F32) {
        if (!q) return p2m_batch_t<float, float, float, float, REFINE_NONE, 0>(plan, a, shape_idx, blocks, counter, w, s);
        return p2m_batch_solve<float, float, 1>(solve, plan, a, shape_idx, blocks, counter, w, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_m2p(const void *plan, const void *pos, pfem_dtype pos_t, int C,
                             const void *mesh, void *vals, pfem_dtype val_t, int blocks,
                             cudaStream_t s)
{
    const BPlanDev *pl = (const BPlanDev *)plan;
    if (val_t == PFEM_F64 && pos_t == PFEM_F64)
        k_m2p_batch<double, double, double><<<blocks, 256, 0, s>>>(pl, (const double *)pos, C, (const double *)mesh, (double *)vals);
    else if (val_t == PFEM_F32 && pos_t == PFEM_F32)
        k_m2p_batch<float, float, float><<<blocks, 256, 0, s>>>(pl, (const float *)pos, C, (const float *)mesh, (float *)vals);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

}  // namespace pfem
