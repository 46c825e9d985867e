// stars.cu -- the star table (startab.cuh): the Delaunay star of every particle, one thread per
// particle, then the particles whose list attempt failed by a region search.
#include <algorithm>
#include <atomic>

#include "internal.h"
#include "startab.cuh"

namespace pfem {

__global__ void __launch_bounds__(STAR_TPB, 6) k_star_list(Bins B, int R0, StarTab t, DevStatus *st)
{
    __shared__ float2 sxy[STAR_KL * STAR_TPB];
    __shared__ unsigned skey[STAR_KL * STAR_TPB];
    __shared__ int ss[STAR_KL * STAR_TPB];
    __shared__ unsigned char sord[STAR_KL * STAR_TPB];
    __shared__ unsigned char sstk[STAR_KL * STAR_TPB];
    const long long v = blockIdx.x * (long long)STAR_TPB + threadIdx.x;
    if (v >= t.N) return;
    const HullList L{sxy + threadIdx.x, skey + threadIdx.x, ss + threadIdx.x, sord + threadIdx.x,
                      sstk + threadIdx.x, STAR_TPB};
    star_list_slot(B, R0, t, v, L, st);
}

// The queued particles, with the radius of B (the launcher passes the widest one): the hull
// attempt for a short queue (lists in shared memory as in k_star_list, 32 x 18 bytes x 64
// threads = 36 KB), then the region search for the stars still queued.
constexpr int RETRY_TPB = 64;
__global__ void __launch_bounds__(RETRY_TPB) k_star_retry_hull(Bins B, int R0, StarTab t, DevStatus *st)
{
    __shared__ float2 sxy[STAR_KL_RETRY * RETRY_TPB];
    __shared__ unsigned skey[STAR_KL_RETRY * RETRY_TPB];
    __shared__ int ss[STAR_KL_RETRY * RETRY_TPB];
    __shared__ unsigned char sord[STAR_KL_RETRY * RETRY_TPB];
    __shared__ unsigned char sstk[STAR_KL_RETRY * RETRY_TPB];
    const HullList L{sxy + threadIdx.x, skey + threadIdx.x, ss + threadIdx.x, sord + threadIdx.x,
                     sstk + threadIdx.x, RETRY_TPB};
    const int n = min(*t.qcount, (int)min(t.N, (long long)0x7fffffff));
    if (!short_queue(n, t.N)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        star_retry_hull_slot(B, R0, t, t.queue[i], L, st);
}

__global__ void __launch_bounds__(64) k_star_retry(Bins B, int R0, StarTab t, DevStatus *st)
{
    const int n = min(*t.qcount, (int)min(t.N, (long long)0x7fffffff));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        star_retry_slot(B, R0, t, t.queue[i], st);
}

size_t star_tab_bytes(long long N)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t n = (size_t)(N > 0 ? N : 1);
    return al(n * KMAX * sizeof(int)) + al(n * sizeof(int)) + al(n * sizeof(int));
}

// A fresh stamp for each table build (1 .. 2^24 - 1, cycling).
unsigned next_tab_gen()
{
    static std::atomic<unsigned> gen{0};
    unsigned g;
    do {
        g = (gen.fetch_add(1, std::memory_order_relaxed) + 1) & 0xffffffu;
    } while (g == 0);
    return g;
}

StarTab star_tab_layout(char *base, long long N, int *qcount)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t n = (size_t)(N > 0 ? N : 1);
    StarTab t;
    t.nbr = (int *)base;
    t.cnt = (int *)(base + al(n * KMAX * sizeof(int)));
    t.queue = (int *)(base + al(n * KMAX * sizeof(int)) + al(n * sizeof(int)));
    t.qcount = qcount;
    t.N = N;
    t.gen = next_tab_gen();
    return t;
}

cudaError_t launch_star_table(const Bins &B, int R0, int rmax_far, const StarTab &t,
                              DevStatus *st, cudaStream_t s)
{
    if (t.N <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(t.qcount, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_star_list<<<(unsigned)((t.N + STAR_TPB - 1) / STAR_TPB), STAR_TPB, 0, s>>>(B, R0, t, st);
    Bins Bf = B;
    Bf.rmax = std::max(B.rmax, rmax_far);
    k_star_retry_hull<<<num_sms() * PFEM_RETRY_BLOCKS, RETRY_TPB, 0, s>>>(Bf, R0, t, st);
    k_star_retry<<<num_sms() * PFEM_RETRY_REGION_BLOCKS, 64, 0, s>>>(Bf, R0, t, st);
    count_launch(3);
    return cudaGetLastError();
}

}  // namespace pfem
