// cells.cu -- particle bins (a stable counting sort by bin), the first two steps of every
// projection: canonicalise positions to 32-bit fixed point and order particles by
// (bin, original index).  The paper locates particles through CGAL (App. A); this replaces
// that with a deterministic bin structure the projection kernels search.
//
// Steps: (1) per particle: fixed point, bin, and an arrival rank inside the bin (atomic
// counter; order not yet deterministic); (2) exclusive scan of the bin counts; (3) scatter to
// slot start + rank; (4) per particle: its rank by original index within its bin, which makes
// the order stable and bit-reproducible; (5) per slot: gather sorted positions and fixed-point
// coordinates (coalesced writes).
#include "internal.h"

namespace pfem {

template <typename P>
__global__ void k_bin(const P *__restrict__ pos, long long N, int nb, int *__restrict__ key,
                      int *__restrict__ rank, int *__restrict__ count)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x) {
        P x, y;
        load_pos(pos, m, x, y);
        const int b = bin_of(fx_of(y), nb) * nb + bin_of(fx_of(x), nb);
        key[m] = b;
        rank[m] = atomicAdd(count + b, 1);
    }
}

__global__ void k_scatter(long long N, const int *__restrict__ key, const int *__restrict__ rank,
                          const int *__restrict__ cell_start, int *__restrict__ perm)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x)
        perm[__ldg(cell_start + key[m]) + rank[m]] = (int)m;
}

// Order each bin's slots by original index: the slot of particle m in bin b is
// cell_start[b] + #{particles of b with a smaller index}.  One thread per particle counts over
// its bin (the scatter left the bin's particles in arrival order), so a crowded bin costs
// parallel work, not a serial sort.
__global__ void k_rank_bins(long long N, const int *__restrict__ key,
                            const int *__restrict__ cell_start, const int *__restrict__ perm,
                            int *__restrict__ sorted)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = perm[i];
        const int b = __ldg(key + m);
        const int s0 = __ldg(cell_start + b), s1 = __ldg(cell_start + b + 1);
        int r = 0;
        for (int j = s0; j < s1; ++j) r += perm[j] < m;
        sorted[s0 + r] = m;
    }
}

// Final order (from k_rank_bins) into perm, and the positions and fixed-point coordinates in
// slot order (coalesced writes).
template <typename P>
__global__ void k_gather(long long N, const P *__restrict__ pos, const int *__restrict__ sorted,
                         int *__restrict__ perm, P *__restrict__ pos_sorted,
                         uint2 *__restrict__ q_sorted)
{
    using V2 = typename Vec2<P>::type;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int m = __ldg(sorted + s);
        perm[s] = m;
        const V2 v = __ldg(reinterpret_cast<const V2 *>(pos) + m);
        reinterpret_cast<V2 *>(pos_sorted)[s] = v;
        q_sorted[s] = make_uint2(fx_of(v.x), fx_of(v.y));
    }
}

// ---------------------------------------------------------------- exclusive scan of int32

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER;

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_tiles(const int *__restrict__ in, int *__restrict__ out, long long n, int *__restrict__ sums)
{
    __shared__ int warp_tot[SCAN_THREADS / 32];
    const long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_PER;
    int v[SCAN_PER];
    int t = 0;
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        t += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    int run = incl - t + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_PER; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = warp_tot[31];
}

__global__ void k_scan_add(int *__restrict__ out, long long n, const int *__restrict__ offs)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += __ldg(offs + i / SCAN_TILE);
}

size_t scan_scratch_ints(long long n)
{
    size_t total = 0;
    while (n > 1) {
        const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
        total += 2 * (size_t)tiles + 64;
        n = tiles;
    }
    return total + 64;
}

// Exclusive scan in -> out (n elements); scratch holds scan_scratch_ints(n) ints.
cudaError_t scan_exclusive(const int *in, int *out, long long n, int *scratch, cudaStream_t s)
{
    const long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int *sums = scratch;
    int *sums_scan = scratch + tiles + 32;
    k_scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums);
    count_launch();
    if (tiles > 1) {
        cudaError_t e = scan_exclusive(sums, sums_scan, tiles, sums_scan + tiles + 32, s);
        if (e != cudaSuccess) return e;
        k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums_scan);
        count_launch();
    }
    return cudaGetLastError();
}

static unsigned grid_for(long long work, int threads)
{
    long long b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > num_sms() * 64LL) b = num_sms() * 64LL;
    return (unsigned)b;
}

// Scatter to slot start + rank, order each bin by original index, gather sorted positions.
template <typename P>
static cudaError_t sort_gather_t(long long nbins, long long N, const P *pos, const int *key,
                                 int *rank, const int *cell_start, int *perm, P *pos_sorted,
                                 uint2 *q_sorted, cudaStream_t s)
{
    if (N > 0) {
        // the arrival ranks are dead after the scatter: their array takes the final order
        int *sorted = rank;
        k_scatter<<<grid_for(N, 256), 256, 0, s>>>(N, key, rank, cell_start, perm);
        k_rank_bins<<<grid_for(N, 256), 256, 0, s>>>(N, key, cell_start, perm, sorted);
        k_gather<P><<<grid_for(N, 256), 256, 0, s>>>(N, pos, sorted, perm, pos_sorted, q_sorted);
        count_launch(3);
    }
    return cudaGetLastError();
}

cudaError_t launch_sort_gather(long long nbins, long long N, const void *pos, pfem_dtype pos_t,
                               const int *key, int *rank, const int *cell_start, int *perm,
                               void *pos_sorted, uint32_t *q_sorted, cudaStream_t s)
{
    if (pos_t == PFEM_F64)
        return sort_gather_t<double>(nbins, N, (const double *)pos, key, rank, cell_start, perm,
                                     (double *)pos_sorted, (uint2 *)q_sorted, s);
    return sort_gather_t<float>(nbins, N, (const float *)pos, key, rank, cell_start, perm,
                                (float *)pos_sorted, (uint2 *)q_sorted, s);
}

template <typename P>
static cudaError_t build_cells_t(int nb, long long N, const P *pos, int *cell_start, int *perm,
                                 P *pos_sorted, uint2 *q_sorted, const WsLayout &L, char *ws,
                                 cudaStream_t s)
{
    const long long nbins = (long long)nb * nb;
    int *count = (int *)(ws + L.count);
    int *key = (int *)(ws + L.key);
    int *rank = (int *)(ws + L.rank);
    int *scr = (int *)(ws + L.scan);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(nbins + 1), s);
    if (e != cudaSuccess) return e;
    if (N > 0) {
        k_bin<P><<<grid_for(N, 256), 256, 0, s>>>(pos, N, nb, key, rank, count);
        count_launch();
    }
    e = scan_exclusive(count, cell_start, nbins + 1, scr, s);
    if (e != cudaSuccess) return e;
    return sort_gather_t<P>(nbins, N, pos, key, rank, cell_start, perm, pos_sorted, q_sorted, s);
}

cudaError_t launch_build_cells(int nb, long long N, const void *pos, pfem_dtype pos_t,
                               int *cell_start, int *perm, void *pos_sorted, uint32_t *q_sorted,
                               const WsLayout &L, void *ws, cudaStream_t s)
{
    if (pos_t == PFEM_F64)
        return build_cells_t<double>(nb, N, (const double *)pos, cell_start, perm,
                                     (double *)pos_sorted, (uint2 *)q_sorted, L, (char *)ws, s);
    return build_cells_t<float>(nb, N, (const float *)pos, cell_start, perm, (float *)pos_sorted,
                                (uint2 *)q_sorted, L, (char *)ws, s);
}

}  // namespace pfem
