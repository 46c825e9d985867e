// advect.cu -- the particle move and the incremental re-binning of the projection loop the paper
// runs on Zalesak's disk (Sec. 3.1: every step projects the field mesh -> particles, moves the
// particles one step with the midpoint velocity, rebuilds the particle shape functions and
// projects back particles -> mesh).
//
// pfem_advect_midpoint: r_half = r + dt/2 u(r), r_new = r + dt u(r_half) (the midpoint scheme of
// Sec. 3.2), with u the mesh velocity field interpolated at the particle by linear FE on the
// structured mesh (the same rule as M2P, eq. m2p).
//
// pfem_update_cells: after such a move most particles stay in their bin and the rest move to
// a neighbouring bin.  The new bins are then filled without atomics from the old ones: the
// particles that end in bin b' come from the 3 x 3 old bins around b', each old bin's slots in
// original-index order, so a particle's rank in b' is the number of particles of those nine
// old bins that end in b' with a smaller original index.  The result is the stable order of
// pfem_build_cells, bit for bit.  A particle that moved further records PFEM_ERR_CAPACITY.
#include "internal.h"

namespace pfem {

template <typename R> __device__ __forceinline__ R cell_coord(R x, int i, int nc)
{
    const R xw = x - floor(x);
    R s = fma(xw, (R)nc, (R)(-i));
    if (s > (R)(0.5 * nc)) s -= (R)nc;                  // fixed point rounded up to 2^32 -> cell 0
    return s;
}

// Linear-FE interpolation of the two velocity components at (x, y) (eq. m2p).
template <typename P>
__device__ __forceinline__ void fe_velocity(int n, const P *__restrict__ mesh, P x, P y, P &u, P &v)
{
    const int nc = n - 1;
    const int i = bin_of(fx_of(x), nc), j = bin_of(fx_of(y), nc);
    const P s = cell_coord<P>(x, i, nc), t = cell_coord<P>(y, j, nc);
    const long long n00 = (long long)j * n + i;
    long long nb_, nc_;
    P w0, w1, w2;
    if (s >= t) { nb_ = n00 + 1; nc_ = n00 + n + 1; w0 = P(1) - s; w1 = s - t; w2 = t; }
    else        { nb_ = n00 + n + 1; nc_ = n00 + n; w0 = P(1) - t; w1 = s; w2 = t - s; }
    u = w0 * __ldg(mesh + 2 * n00) + w1 * __ldg(mesh + 2 * nb_) + w2 * __ldg(mesh + 2 * nc_);
    v = w0 * __ldg(mesh + 2 * n00 + 1) + w1 * __ldg(mesh + 2 * nb_ + 1) + w2 * __ldg(mesh + 2 * nc_ + 1);
}

template <typename P>
__global__ void __launch_bounds__(256) k_advect_midpoint(int n, long long N, const P *__restrict__ pos,
                                                         const P *__restrict__ vel, P dt,
                                                         P *__restrict__ out)
{
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N;
         m += (long long)gridDim.x * blockDim.x) {
        P x, y, u, v;
        load_pos(pos, m, x, y);
        fe_velocity(n, vel, x, y, u, v);
        const P xh = x + (P)0.5 * dt * u, yh = y + (P)0.5 * dt * v;
        fe_velocity(n, vel, xh, yh, u, v);
        const P xn = x + dt * u, yn = y + dt * v;
        out[2 * m] = xn - floor(xn);
        out[2 * m + 1] = yn - floor(yn);
    }
}

cudaError_t launch_advect_midpoint(int n, long long N, const void *pos, pfem_dtype pos_t,
                                   const void *vel, double dt, void *out, cudaStream_t s)
{
    long long blocks = (N + 255) / 256;
    if (blocks > num_sms() * 16LL) blocks = num_sms() * 16LL;
    if (blocks < 1) blocks = 1;
    if (pos_t == PFEM_F64)
        k_advect_midpoint<double><<<(unsigned)blocks, 256, 0, s>>>(
            n, N, (const double *)pos, (const double *)vel, dt, (double *)out);
    else
        k_advect_midpoint<float><<<(unsigned)blocks, 256, 0, s>>>(
            n, N, (const float *)pos, (const float *)vel, (float)dt, (float *)out);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- incremental re-binning

// Bin of a fixed-point pair on the nb x nb grid, and whether it lies within one bin (on the
// torus) of the old bin (obx, oby).
__device__ __forceinline__ int wrap_delta(int d, int nb)
{
    d = d > nb / 2 ? d - nb : d;
    return d < -nb / 2 ? d + nb : d;
}

// Per old slot: the particle's new fixed point and new bin; a move beyond the neighbouring bins
// records PFEM_ERR_CAPACITY (detail: the particle's original index).
template <typename P>
__global__ void __launch_bounds__(256) k_upd_bin(long long N, int nb, const P *__restrict__ pos,
                                                 const int *__restrict__ perm_old,
                                                 const uint2 *__restrict__ q_old,
                                                 int *__restrict__ newbin, uint2 *__restrict__ qnew,
                                                 DevStatus *st)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int m = __ldg(perm_old + s);
        P x, y;
        load_pos(pos, m, x, y);
        const uint2 q = make_uint2(fx_of(x), fx_of(y));
        const uint2 qo = __ldg(q_old + s);
        const int bx = bin_of(q.x, nb), by = bin_of(q.y, nb);
        const int dx = wrap_delta(bx - bin_of(qo.x, nb), nb), dy = wrap_delta(by - bin_of(qo.y, nb), nb);
        if (dx < -1 || dx > 1 || dy < -1 || dy > 1) record_error(st, PFEM_ERR_CAPACITY, m);
        newbin[s] = by * nb + bx;
        qnew[s] = q;
    }
}

// Visit the old slots of the 3 x 3 old bins around bin (bx, by): f(slot).
template <typename F>
__device__ __forceinline__ void for_old_neighbours(const int *__restrict__ start_old, int nb, int bx,
                                                   int by, F &&f)
{
    for (int dy = -1; dy <= 1; ++dy) {
        int y = by + dy;
        y += y < 0 ? nb : 0;
        y -= y >= nb ? nb : 0;
        for (int dx = -1; dx <= 1; ++dx) {
            int x = bx + dx;
            x += x < 0 ? nb : 0;
            x -= x >= nb ? nb : 0;
            const int b = y * nb + x;
            const int e = __ldg(start_old + b + 1);
            for (int t = __ldg(start_old + b); t < e; ++t) f(t);
        }
    }
}

// Per new bin: how many particles end in it.
__global__ void __launch_bounds__(256) k_upd_count(int nb, const int *__restrict__ start_old,
                                                   const int *__restrict__ newbin,
                                                   int *__restrict__ count)
{
    const long long nbins = (long long)nb * nb;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbins;
         b += (long long)gridDim.x * blockDim.x) {
        int c = 0;
        for_old_neighbours(start_old, nb, (int)(b % nb), (int)(b / nb),
                           [&](int t) { c += __ldg(newbin + t) == (int)b; });
        count[b] = c;
    }
}

// Per old slot: its new slot = start of its new bin + the number of particles that end in the
// same bin with a smaller original index; write the permutation, sorted positions and fixed
// point there.
template <typename P>
__global__ void __launch_bounds__(256) k_upd_place(long long N, int nb, const P *__restrict__ pos,
                                                   const int *__restrict__ start_old,
                                                   const int *__restrict__ perm_old,
                                                   const int *__restrict__ newbin,
                                                   const uint2 *__restrict__ qnew,
                                                   const int *__restrict__ start_new,
                                                   int *__restrict__ perm, P *__restrict__ pos_sorted,
                                                   uint2 *__restrict__ q_sorted)
{
    using V2 = typename Vec2<P>::type;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        const int b = __ldg(newbin + s), m = __ldg(perm_old + s);
        int r = 0;
        for_old_neighbours(start_old, nb, b % nb, b / nb, [&](int t) {
            r += __ldg(newbin + t) == b && __ldg(perm_old + t) < m;
        });
        const int slot = __ldg(start_new + b) + r;
        perm[slot] = m;
        reinterpret_cast<V2 *>(pos_sorted)[slot] = __ldg(reinterpret_cast<const V2 *>(pos) + m);
        q_sorted[slot] = __ldg(qnew + s);
    }
}

// Workspace of pfem_update_cells: status block, new bins [N], new fixed point [N], bin counts
// and scan scratch.
size_t update_ws_bytes(long long nbins, long long N)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t n = (size_t)(N > 0 ? N : 1);
    return 256 + al(4 * n) + al(8 * n) + al(4 * (size_t)(nbins + 1)) +
           al(4 * scan_scratch_ints(nbins + 1));
}

cudaError_t launch_update_cells(int nb, long long N, const void *pos, pfem_dtype pos_t,
                                const int *start_old, const int *perm_old, const uint32_t *q_old,
                                int *cell_start, int *perm, void *pos_sorted, uint32_t *q_sorted,
                                void *ws, cudaStream_t s)
{
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const long long nbins = (long long)nb * nb;
    const size_t n = (size_t)(N > 0 ? N : 1);
    char *W = (char *)ws;
    DevStatus *st = (DevStatus *)W;
    int *newbin = (int *)(W + 256);
    uint2 *qnew = (uint2 *)(W + 256 + al(4 * n));
    int *count = (int *)(W + 256 + al(4 * n) + al(8 * n));
    int *scr = (int *)(W + 256 + al(4 * n) + al(8 * n) + al(4 * (size_t)(nbins + 1)));
    auto grid = [](long long work) {
        long long b = (work + 255) / 256;
        if (b > num_sms() * 32LL) b = num_sms() * 32LL;
        return (unsigned)(b < 1 ? 1 : b);
    };
    if (N > 0) {
        if (pos_t == PFEM_F64)
            k_upd_bin<double><<<grid(N), 256, 0, s>>>(N, nb, (const double *)pos, perm_old,
                                                      (const uint2 *)q_old, newbin, qnew, st);
        else
            k_upd_bin<float><<<grid(N), 256, 0, s>>>(N, nb, (const float *)pos, perm_old,
                                                     (const uint2 *)q_old, newbin, qnew, st);
        count_launch();
    }
    k_upd_count<<<grid(nbins), 256, 0, s>>>(nb, start_old, newbin, count);
    count_launch();
    cudaError_t e = cudaMemsetAsync(count + nbins, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    e = scan_exclusive(count, cell_start, nbins + 1, scr, s);
    if (e != cudaSuccess || N == 0) return e;
    if (pos_t == PFEM_F64)
        k_upd_place<double><<<grid(N), 256, 0, s>>>(N, nb, (const double *)pos, start_old, perm_old,
                                                    newbin, qnew, cell_start, perm,
                                                    (double *)pos_sorted, (uint2 *)q_sorted);
    else
        k_upd_place<float><<<grid(N), 256, 0, s>>>(N, nb, (const float *)pos, start_old, perm_old,
                                                   newbin, qnew, cell_start, perm,
                                                   (float *)pos_sorted, (uint2 *)q_sorted);
    count_launch();
    return cudaGetLastError();
}

}  // namespace pfem
