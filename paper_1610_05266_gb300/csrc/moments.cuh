// moments.cuh -- the per-edge coefficient system of the quadratically consistent shape
// functions (App. B, eqs. A0, A1, condquad; App. A: minimum-norm solution).
//
// For a Delaunay edge e = (nu, sigma) with stencil S_e, the coefficients A_mu (mu in S_e)
// must satisfy sum A = 0, sum r A = 0 and sum r r^T A = -(1/2)(r_nu - r_sigma)(r_nu - r_sigma)^T
// (eq. condquad rewritten with eqs. A0-A1, eq. A2_2).  In coordinates centred at the edge
// midpoint and scaled by the edge length (the solution does not depend on the frame), with
// p_mu = [1, x, y, x^2, xy, y^2], that is P A = b, P = [p_mu] (6 x k), and the minimum-norm
// solution is A_mu = p_mu . y with M y = b, M = sum_mu p_mu p_mu^T (6 x 6, SPD for a stencil
// not on one conic).  M is factorised by an unrolled Cholesky held in registers.
#pragma once

#include "common.cuh"

namespace pfem {

// packed lower triangle of a symmetric 6x6 matrix: (r, c), r >= c
__host__ __device__ constexpr int tri_ix(int r, int c) { return r * (r + 1) / 2 + c; }

template <typename S> struct Moment {
    S m[21];

    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 21; ++i) m[i] = S(0);
    }

    // M += p p^T for p = [1, x, y, x^2, xy, y^2]
    __device__ __forceinline__ void add(S x, S y)
    {
        const S p[6] = {S(1), x, y, x * x, x * y, y * y};
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) m[tri_ix(r, c)] = fma(p[r], p[c], m[tri_ix(r, c)]);
    }

    // In-place Cholesky M = L L^T; returns false when a pivot is not clearly positive
    // (stencil numerically on one conic: the moment system is rank deficient).
    __device__ __forceinline__ bool factor(S rel_tol)
    {
        S tr = S(0);
#pragma unroll
        for (int r = 0; r < 6; ++r) tr += m[tri_ix(r, r)];
        const S tol = rel_tol * tr;
        bool ok = true;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            S s = m[tri_ix(j, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) s = fma(-m[tri_ix(j, k)], m[tri_ix(j, k)], s);
            ok &= s > tol;
            const S d = sqrt(s > tol ? s : tol);
            const S inv = S(1) / d;
            m[tri_ix(j, j)] = inv;               // store the reciprocal of the pivot
#pragma unroll
            for (int i = j + 1; i < 6; ++i) {
                S t = m[tri_ix(i, j)];
#pragma unroll
                for (int k = 0; k < j; ++k) t = fma(-m[tri_ix(i, k)], m[tri_ix(j, k)], t);
                m[tri_ix(i, j)] = t * inv;
            }
        }
        return ok;
    }

    // Solve L L^T y = b with the factor from factor().
    __device__ __forceinline__ void solve(const S b[6], S y[6]) const
    {
        S z[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            S t = b[r];
#pragma unroll
            for (int k = 0; k < r; ++k) t = fma(-m[tri_ix(r, k)], z[k], t);
            z[r] = t * m[tri_ix(r, r)];
        }
#pragma unroll
        for (int r = 5; r >= 0; --r) {
            S t = z[r];
#pragma unroll
            for (int k = r + 1; k < 6; ++k) t = fma(-m[tri_ix(k, r)], y[k], t);
            y[r] = t * m[tri_ix(r, r)];
        }
    }
};

// ----------------------------------------------------------------- float-float arithmetic
// An unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits), built from the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2): the FP32 sum and
// product of two floats are exact once their rounding error is carried along.  Used for the
// residual of the refined FP32 solve, which must be formed in about twice the working
// precision; on sm_103a FP32 instructions issue at 64 times the rate of FP64 ones.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF ff_two_prod(float a, float b)
{
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ FF ff_norm(float h, float l)
{
    const float s = h + l;
    return {s, l - (s - h)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const FF s = ff_two_sum(a.h, b.h);
    return ff_norm(s.h, s.l + (a.l + b.l));
}

// (a.h + a.l) * b for a float b
__device__ __forceinline__ FF ff_mul(FF a, float b)
{
    const FF p = ff_two_prod(a.h, b);
    return ff_norm(p.h, fmaf(a.l, b, p.l));
}

// (a.h + a.l) * (b.h + b.l)
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const FF p = ff_two_prod(a.h, b.h);
    return ff_norm(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }

// Exact FP32 -> FP64 widening by integer operations on the bit patterns (sign; exponent
// rebiased by 1023 - 127 = 896; the 23 mantissa bits at the top of the 52).  FP32 subnormals
// (below 1.2e-38) become zero.  On sm_103a the format conversion instructions share the
// narrow FP64 pipe, while these run on the integer pipes.
__device__ __forceinline__ double f64_of(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned sign = u & 0x80000000u;
    const unsigned hi = e ? sign | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu) : sign;
    const unsigned lo = e ? u << 29 : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 by truncating the mantissa (relative error below 2^-23), for finite values
// below FP32's largest; magnitudes below FP32's normal range become zero.
__device__ __forceinline__ float f32_trunc(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned u = (hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    return e > 0 ? __uint_as_float(u) : 0.0f;
}

// Refinement of the FP32 moment solve: 0 = none, 1 = residual in FP64, 2 = residual in
// float-float.
enum { REFINE_NONE = 0, REFINE_F64 = 1, REFINE_FF = 2 };

template <typename S> struct SolveTol;
template <> struct SolveTol<double> { static constexpr double v = 1e-13; };
template <> struct SolveTol<float> { static constexpr float v = 1e-6f; };

// Pivot tolerance (relative to the trace) of the fused P2M's Cholesky solve, which hands a
// system below it to the FP64 SVD pass: the normal equations square the stencil's condition,
// so a system is solved fast only while that keeps the precision's accuracy.  Jittered lattices
// stay far above both (smallest pivot 3e-3 of the trace at jitter 0.3); on uniform random
// particles about 0.6 % of the nodes fall below the FP32 value.
#ifndef PFEM_FAST_TOL32
#define PFEM_FAST_TOL32 3e-4f
#endif
#ifndef PFEM_FAST_TOL64
#define PFEM_FAST_TOL64 1e-6
#endif
template <typename S> struct FastTol;
template <> struct FastTol<double> { static constexpr double v = PFEM_FAST_TOL64; };
template <> struct FastTol<float> { static constexpr float v = PFEM_FAST_TOL32; };

}  // namespace pfem
