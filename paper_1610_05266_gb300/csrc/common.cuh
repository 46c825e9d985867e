// common.cuh -- shared device helpers of libpfem: fixed-point topology coordinates,
// bins, the device status word and dtype-generic loads/stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pfem.h"

namespace pfem {

// ----------------------------------------------------------------- status word
// Layout of the first 256 bytes of every workspace: the status code, an error count and the
// index of the first failure.  Device code records the first error and never traps.
struct DevStatus {
    int32_t code;
    int32_t count;
    long long detail;
};

__device__ inline void record_error(DevStatus *st, int code, long long detail)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
    atomicAdd(&st->count, 1);
}

// ----------------------------------------------------------------- fixed point
// q = round_half_even(x * 2^32) mod 2^32.  The scaling by 2^32 is exact in both precisions.
__device__ __forceinline__ uint32_t fx_of(float x)
{
    return (uint32_t)(unsigned long long)__float2ll_rn(x * 4294967296.0f);
}
__device__ __forceinline__ uint32_t fx_of(double x)
{
    return (uint32_t)(unsigned long long)__double2ll_rn(x * 4294967296.0);
}

// Fixed-point coordinate of mesh node I (0 <= I < nc): round(I * 2^32 / nc).
__host__ __device__ __forceinline__ uint32_t node_fx(int I, int nc)
{
    return (uint32_t)((((unsigned long long)I << 32) + (unsigned long long)(nc / 2)) /
                      (unsigned long long)nc);
}

// Bin of a fixed-point coordinate on an nb-per-side grid: (q * nb) >> 32.
__device__ __forceinline__ int bin_of(uint32_t q, int nb) { return (int)__umulhi(q, (uint32_t)nb); }

// First fixed-point coordinate of bin b (0 <= b <= nb): ceil(b * 2^32 / nb).
__device__ __forceinline__ long long bin_lo(int b, int nb)
{
    return (long long)((((unsigned long long)b << 32) + (unsigned long long)(nb - 1)) /
                       (unsigned long long)nb);
}

// ----------------------------------------------------------------- dtype helpers
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(float v) { return v; }

template <typename S, typename R> __device__ __forceinline__ R load_val(const S *p) { return (R)p[0]; }
template <> __device__ __forceinline__ float load_val<__nv_bfloat16, float>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_val<float, float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ double load_val<double, double>(const double *p) { return __ldg(p); }

template <typename S, typename R> __device__ __forceinline__ void store_val(S *p, R v) { p[0] = (S)v; }
template <> __device__ __forceinline__ void store_val<__nv_bfloat16, float>(__nv_bfloat16 *p, float v)
{
    p[0] = __float2bfloat16_rn(v);
}

// Position pair of slot s.
template <typename P> __device__ __forceinline__ void load_pos(const P *pos, long long s, P &x, P &y)
{
    typename Vec2<P>::type v = __ldg(reinterpret_cast<const typename Vec2<P>::type *>(pos) + s);
    x = v.x;
    y = v.y;
}

// Minimal image of a coordinate difference on the unit torus.
__device__ __forceinline__ double wrap1(double d) { return d - rint(d); }
__device__ __forceinline__ float wrap1(float d) { return d - rintf(d); }

}  // namespace pfem
