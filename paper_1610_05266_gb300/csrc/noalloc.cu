// noalloc.cu -- pfem_build_cells_noalloc: the particle binning of pfem_build_cells for callers
// that cannot hand the library a workspace.
//
// Some callers cannot allocate device memory at the point where they need the bins: code
// running inside a host application that owns every device allocation (a simulation driver
// calling a plug-in from its time-step callback), real-time loops that must not take the
// device-wide synchronisation a cudaMalloc/cudaFree can imply, or hosts whose memory pool is
// fixed up front.  This entry point uses a fixed scratch area compiled into the library
// instead of a caller workspace.  The caller still provides every input and output buffer.
//
// The scratch is a file-scope __device__ array: every GPU on which this library's module is
// loaded holds it until the process exits.  Host code cannot pass the array's name to a
// kernel (on the host it is only a stand-in for the symbol), so the device address is looked
// up once per device with cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "internal.h"

namespace pfem {

constexpr long long NOALLOC_MAX_N = 1LL << 22;        // 4,194,304 particles
constexpr long long NOALLOC_MAX_BINS = 1LL << 20;     // nb <= 1024 bins per side

// Bytes the scratch must hold: the build_cells workspace layout at the maximum sizes.
constexpr size_t noalloc_bytes()
{
    // 256 (status) + counts (bins+1) + key (N) + rank (N) + scan scratch, each 256-aligned;
    // scan scratch for 2^20+1 elements is below 2*(257+1)+3*64 ints.
    return 256 + (((size_t)(NOALLOC_MAX_BINS + 1) * 4 + 255) & ~(size_t)255) +
           2 * (((size_t)NOALLOC_MAX_N * 4 + 255) & ~(size_t)255) + 8192;
}

static __device__ __align__(256) unsigned char g_noalloc_scratch[noalloc_bytes()];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[64];

// Device address of the scratch on the current device (looked up on first use per device).
static cudaError_t noalloc_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace pfem

extern "C" pfem_status pfem_build_cells_noalloc(int32_t nb, int64_t N, const void *pos,
                                                pfem_dtype pos_t, int32_t *cell_start,
                                                int32_t *perm, void *pos_sorted,
                                                uint32_t *q_sorted, void *stream)
{
    using namespace pfem;
    if (nb < 1 || N < 0) return PFEM_ERR_INVALID_ARG;
    if ((long long)nb * nb > NOALLOC_MAX_BINS || N > NOALLOC_MAX_N) return PFEM_ERR_CAPACITY;
    if (!cell_start || (N > 0 && (!pos || !perm || !pos_sorted || !q_sorted)))
        return PFEM_ERR_INVALID_ARG;
    if (pos_t != PFEM_F64 && pos_t != PFEM_F32) return PFEM_ERR_INVALID_ARG;
    const WsLayout L = ws_layout(0, nb, N, 1);
    if (L.total > noalloc_bytes()) return PFEM_ERR_CAPACITY;
    void *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return PFEM_ERR_CUDA;
    // launch_build_cells zeroes the bin counters it accumulates into before using them.
    e = launch_build_cells(nb, N, pos, pos_t, cell_start, perm, pos_sorted, q_sorted, L, scratch,
                           (cudaStream_t)stream);
    return e == cudaSuccess ? PFEM_OK : PFEM_ERR_CUDA;
}
