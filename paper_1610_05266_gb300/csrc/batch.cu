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

struct BPlanDev {
    int P;
    int pad;
    long long n_items[BT_SHAPES];
    long long n_chunks;
    long long total_bins;
    // followed in memory by: BDesc desc[P]; long long tile_prefix[BT_SHAPES][P+1];
    // long long chunk_prefix[P+1]
};

__host__ __device__ inline size_t plan_bytes(int P)
{
    return sizeof(BPlanDev) + sizeof(BDesc) * (size_t)P +
           sizeof(long long) * (size_t)(BT_SHAPES + 1) * (size_t)(P + 1);
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

template <typename P, typename V, typename R, typename S, bool REFINE, int SHAPE>
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
        P2MArgs a = base;
        a.n = d.n;
        a.B.start = base.B.start + d.boff;
        a.B.nb = d.nb;
        a.B.rmax = d.rmax;
        a.B.dmax = d.dmax;
        a.R0 = d.R0;
        a.out = (void *)((V *)base.out + d.noff * base.C);
        p2m_node<P, V, R, S, REFINE, SHAPE, false>(a, I, J);
    }
}

// The quadratic P2M with FP32 solves in two kernels, as for one problem: this persistent kernel
// writes every node's record (at its problem's node offset, with its coordinates), then
// k_p2m_solve runs over all nodes of the batch.
template <typename P, typename V, typename R>
__global__ void __launch_bounds__(256, PFEM_GEOM_MIN_BLOCKS / 2) k_p2m_batch_geom(
    const BPlanDev *pl, int shape_idx, P2MArgs base, unsigned long long *counter, NodeRecs r)
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
        P2MArgs a = base;
        a.n = d.n;
        a.B.start = base.B.start + d.boff;
        a.B.nb = d.nb;
        a.B.rmax = d.rmax;
        a.B.dmax = d.dmax;
        a.R0 = d.R0;
        a.out = (void *)((V *)base.out + d.noff * base.C);
        geom_node<P, V, R>(a, r, I, J, d.noff + (long long)J * d.n + I);
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
    pl->P = P;
    long long poff = 0, boff = 0, noff = 0;
    const int TYs[BT_SHAPES] = {4, 8, 16};
    for (int s = 0; s < BT_SHAPES; ++s) tiles[(long long)s * (P + 1)] = 0;
    chunks[0] = 0;
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
    }
    if (poff >= (1LL << 31) || boff >= (1LL << 31)) return PFEM_ERR_INVALID_ARG;
    for (int s = 0; s < BT_SHAPES; ++s) pl->n_items[s] = tiles[(long long)s * (P + 1) + P];
    pl->n_chunks = chunks[P];
    pl->total_bins = boff;
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
        k_bin_batch<double><<<152 * 8, 256, 0, s>>>(pl, (const double *)pos, key, rank, count);
    else
        k_bin_batch<float><<<152 * 8, 256, 0, s>>>(pl, (const float *)pos, key, rank, count);
    count_launch();
    e = scan_exclusive(count, cell_start, bins_total + 1, (int *)(W + L.scan), s);
    if (e != cudaSuccess) return e;
    return launch_sort_gather(bins_total, Ntot, pos, pos_t, key, rank, cell_start, perm, pos_sorted,
                              q_sorted, s);
}

template <typename P, typename V, typename R, typename S, bool REF, int SHAPE>
static cudaError_t p2m_batch_t(const void *plan, const P2MArgs &base, int shape_idx, int blocks,
                               unsigned long long *counter, const NodeRecs *rec, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int TYs[BT_SHAPES] = {4, 8, 16};
    if (SHAPE == PFEM_SHAPE_QUADRATIC && sizeof(S) == sizeof(float) && rec) {
        k_p2m_batch_geom<P, V, R><<<blocks, 16 * TYs[shape_idx], 0, s>>>(
            (const BPlanDev *)plan, shape_idx, base, counter, *rec);
        k_p2m_solve<P, V, R, S, REF><<<(unsigned)((rec->nodes + 127) / 128), 128, 0, s>>>(base, *rec);
        count_launch(2);
        return cudaGetLastError();
    }
    k_p2m_batch<P, V, R, S, REF, SHAPE><<<blocks, 16 * TYs[shape_idx], 0, s>>>(
        (const BPlanDev *)plan, shape_idx, base, counter);
    count_launch();
    return cudaGetLastError();
}

// Workspace of the batched P2M: status (byte 0) and work counter (byte 64), then the node
// records of the two-kernel path from byte 256.
size_t batch_p2m_ws_bytes(long long nodes_total)
{
    NodeRecs r;
    return 256 + node_recs_layout(nullptr, nodes_total, &r, true);
}

cudaError_t launch_batch_p2m(const void *plan, const void *pos_sorted, const uint32_t *q_sorted,
                             const int *cell_start, const int *perm, int C, const void *vals,
                             pfem_dtype val_t, pfem_shape shape, pfem_solve solve, void *mesh,
                             int shape_idx, int blocks, long long nodes_total, void *ws,
                             size_t ws_bytes, cudaStream_t s)
{
    NodeRecs recs;
    const NodeRecs *rec = nullptr;
    if (nodes_total > 0 && ws_bytes >= batch_p2m_ws_bytes(nodes_total)) {
        node_recs_layout((char *)ws + 256, nodes_total, &recs, true);
        rec = &recs;
    }
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
    unsigned long long *counter = (unsigned long long *)((char *)ws + 64);
    const bool q = shape == PFEM_SHAPE_QUADRATIC;
    if (val_t == PFEM_F64) {
        if (!q) return p2m_batch_t<double, double, double, double, false, 0>(plan, a, shape_idx, blocks, counter, rec, s);
        return p2m_batch_t<double, double, double, double, false, 1>(plan, a, shape_idx, blocks, counter, rec, s);
    }
    if (val_t == PFEM_F32) {
        if (!q) return p2m_batch_t<float, float, float, float, false, 0>(plan, a, shape_idx, blocks, counter, rec, s);
        if (solve == PFEM_SOLVE_F64) return p2m_batch_t<float, float, float, double, false, 1>(plan, a, shape_idx, blocks, counter, rec, s);
        if (solve == PFEM_SOLVE_F32) return p2m_batch_t<float, float, float, float, false, 1>(plan, a, shape_idx, blocks, counter, rec, s);
        return p2m_batch_t<float, float, float, float, true, 1>(plan, a, shape_idx, blocks, counter, rec, s);
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
