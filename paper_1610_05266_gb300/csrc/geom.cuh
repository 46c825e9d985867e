// geom.cuh -- local Delaunay geometry on the GPU (App. B: Delaunay triangulation of the
// particles, whose edges define "neighbours"; linear FE shape functions on its triangles).
//
// Nothing here builds a global triangulation.  A thread computes the Delaunay star of one
// particle by gift-wrapping over the particles of the bins around it, and certifies every
// triangle it returns by checking that the triangle's circumcircle lies inside the searched
// region (so no particle outside it can be inside the circle); otherwise the region grows.
//
// Predicates are exact on 32-bit fixed-point coordinates (differences as signed 32-bit ints
// give the minimal image on the torus): orientation in 64-bit integers; incircle first in
// FP32 with a forward error bound, and in 128-bit integers when the filter cannot decide.
// Ties (four cocircular particles) are broken by perturbing the lifted heights, the particle
// with the largest key (qy << 32 | qx) taking the dominant perturbation.
#pragma once

#include "common.cuh"

namespace pfem {

constexpr int KMAX = PFEM_KMAX;

// Internal result of a search that ran out of its region (bins up to rmax) before it could
// certify its answer: the caller queues the node for a pass with a wider radius.  Not a public
// status; it becomes PFEM_ERR_CAPACITY where no wider pass follows.
constexpr int PFEM_FAR = 65;

struct Bins {
    const uint2 *__restrict__ q;      // [N] fixed-point (x, y) in slot order
    const int *__restrict__ start;    // [nb*nb + 1]
    int nb;
    int rmax;                         // largest search radius (bins) tried before giving up
    float dmax;                       // candidate distance cutoff of the first attempt (fixed point)
    int kcap = KMAX;                  // largest star kept (<= KMAX); larger: PFEM_ERR_CAPACITY
    int walk_cap = 64;                // visibility-walk steps before PFEM_ERR_TIMEOUT
};

__device__ __forceinline__ int2 rel(uint2 a, uint2 o)
{
    return make_int2((int)(a.x - o.x), (int)(a.y - o.y));
}

__device__ __forceinline__ unsigned long long key_of(uint2 q)
{
    return ((unsigned long long)q.y << 32) | q.x;
}

// a x b for relative coordinates (|components| < 2^30): exact in 64 bits.
__device__ __forceinline__ long long cross(int2 a, int2 b)
{
    return (long long)a.x * b.y - (long long)a.y * b.x;
}

// Orientation of (a, b, c) given relative to a common origin: (b - a) x (c - a).
__device__ __forceinline__ long long orient3(int2 a, int2 b, int2 c)
{
    int2 u = make_int2(b.x - a.x, b.y - a.y), w = make_int2(c.x - a.x, c.y - a.y);
    return cross(u, w);
}

// A region: bins [bx-R, bx+R] x [by-R, by+R] around the bin of a point, and the guaranteed
// clearance from that point to the region's edge on each side (fixed-point units).
struct Region {
    int bx, by, R;
    float cl_lo_x, cl_hi_x, cl_lo_y, cl_hi_y;
};

__device__ __forceinline__ Region make_region(const Bins &B, uint2 p, int R)
{
    Region g;
    g.R = R;
    // q * nb = b * 2^32 + f: bin b, and p lies f / nb fixed-point units past the bin's real
    // left edge (b * 2^32 / nb).  The integer bin boundaries are within one unit of the real
    // ones, so the clearances below, reduced by a relative 2^-20 and 4 units for the FP32
    // rounding, are lower bounds of the exact ones.
    const float inv = __frcp_rn((float)B.nb);
    const float w = 4294967296.0f * inv;
    const unsigned long long mx = (unsigned long long)p.x * (unsigned)B.nb;
    const unsigned long long my = (unsigned long long)p.y * (unsigned)B.nb;
    g.bx = (int)(mx >> 32);
    g.by = (int)(my >> 32);
    const float lx = (float)(unsigned)mx * inv, ly = (float)(unsigned)my * inv;
    const float Rw = (float)R * w, s = 1.0f - 9.5367431640625e-07f;
    g.cl_lo_x = fmaf(lx + Rw, s, -4.f);
    g.cl_hi_x = fmaf((w - lx) + Rw, s, -4.f);
    g.cl_lo_y = fmaf(ly + Rw, s, -4.f);
    g.cl_hi_y = fmaf((w - ly) + Rw, s, -4.f);
    return g;
}

// Visit every slot of the region's bins once (rows are contiguous slot ranges unless they
// wrap around the torus).
template <typename F>
__device__ __forceinline__ void for_region(const Bins &B, const Region &g, F &&f)
{
    const int nb = B.nb;
    for (int dy = -g.R; dy <= g.R; ++dy) {
        int by = g.by + dy;
        by += by < 0 ? nb : 0;
        by -= by >= nb ? nb : 0;
        const int *row = B.start + (long long)by * nb;
        int x0 = g.bx - g.R, x1 = g.bx + g.R;       // inclusive
        if (x0 >= 0 && x1 < nb) {
            int s1 = __ldg(row + x1 + 1);
            for (int s = __ldg(row + x0); s < s1; ++s) f(s);
        } else {
            int a0 = x0 < 0 ? x0 + nb : x0;          // wrapped first run: [a0, nb)
            int a1 = x1 >= nb ? x1 - nb : x1;        // second run: [0, a1]
            if (x0 < 0) {
                int s1 = __ldg(row + nb);
                for (int s = __ldg(row + a0); s < s1; ++s) f(s);
                int t1 = __ldg(row + x1 + 1);
                for (int s = __ldg(row); s < t1; ++s) f(s);
            } else {
                int s1 = __ldg(row + nb);
                for (int s = __ldg(row + x0); s < s1; ++s) f(s);
                int t1 = __ldg(row + a1 + 1);
                for (int s = __ldg(row); s < t1; ++s) f(s);
            }
        }
    }
}

// The region's slots as contiguous runs f(first, end) (one per row, two where a row wraps).
template <typename F>
__device__ __forceinline__ void for_region_runs(const Bins &B, const Region &g, F &&f)
{
    const int nb = B.nb;
    for (int dy = -g.R; dy <= g.R; ++dy) {
        int by = g.by + dy;
        by += by < 0 ? nb : 0;
        by -= by >= nb ? nb : 0;
        const int *row = B.start + (long long)by * nb;
        const int x0 = g.bx - g.R, x1 = g.bx + g.R;       // inclusive
        if (x0 >= 0 && x1 < nb) {
            f(__ldg(row + x0), __ldg(row + x1 + 1));
        } else if (x0 < 0) {
            f(__ldg(row + x0 + nb), __ldg(row + nb));
            f(__ldg(row), __ldg(row + x1 + 1));
        } else {
            f(__ldg(row + x0), __ldg(row + nb));
            f(__ldg(row), __ldg(row + x1 - nb + 1));
        }
    }
}

// Circle through the origin v and points a, b (v, a, b counter-clockwise), as the lifted
// determinant det3(c) = K |c|^2 + P cx + Q cy: c is strictly inside iff det3(c) < 0.
// P, Q are rounded to FP32; Pa, Qa bound the magnitudes of the terms they were formed from.
struct Circ {
    float K, P, Q, Pa, Qa;
};

__device__ __forceinline__ Circ make_circ(int2 a, int2 b)
{
    Circ c;
    const long long la = (long long)a.x * a.x + (long long)a.y * a.y;
    const long long lb = (long long)b.x * b.x + (long long)b.y * b.y;
    const float fla = (float)la, flb = (float)lb;
    const float t1 = flb * (float)a.y, t2 = fla * (float)b.y;
    const float t3 = fla * (float)b.x, t4 = flb * (float)a.x;
    c.K = (float)cross(a, b);
    c.P = t1 - t2;
    c.Pa = fabsf(t1) + fabsf(t2);
    c.Q = t3 - t4;
    c.Qa = fabsf(t3) + fabsf(t4);
    return c;
}

// FP32 filter: +1 strictly inside, -1 strictly outside, 0 undecided.  The bound 2^-20 (16
// units of FP32 rounding) times the sum of absolute terms covers the rounding of the inputs,
// of K, P, Q and of the evaluation (at most about 8 roundings on any path).
__device__ __forceinline__ int circ_filter(const Circ &c, int2 p)
{
    const float x = (float)p.x, y = (float)p.y;
    const float l = fmaf(x, x, y * y);
    const float det = fmaf(c.K, l, fmaf(c.P, x, c.Q * y));
    const float mag = fmaf(c.K, l, fmaf(c.Pa, fabsf(x), c.Qa * fabsf(y)));
    const float bound = 9.5367431640625e-07f * mag;
    return det < -bound ? 1 : (det > bound ? -1 : 0);
}

// Exact incircle with the tie-break.  Points are relative to v (the origin); qv, qa, qb, qc
// are the absolute fixed-point coordinates that give the keys.  Returns +1 when c is inside
// circle(v, a, b) (perturbed), -1 otherwise.
static __device__ __noinline__ int incircle_exact(int2 a, int2 b, int2 c, uint2 qv, uint2 qa,
                                           uint2 qb, uint2 qc)
{
    const long long la = (long long)a.x * a.x + (long long)a.y * a.y;
    const long long lb = (long long)b.x * b.x + (long long)b.y * b.y;
    const long long lc = (long long)c.x * c.x + (long long)c.y * c.y;
    const __int128 det = (__int128)la * cross(b, c) - (__int128)lb * cross(a, c) +
                         (__int128)lc * cross(a, b);
    if (det < 0) return 1;
    if (det > 0) return -1;
    // Lifting v, a, b or c by the dominant infinitesimal changes the lifted 4x4 determinant
    // (positive inside) by the cofactor of that point: orient(a,b,c), -orient(v,b,c),
    // orient(v,a,c), -orient(v,a,b) respectively.
    const unsigned long long kv = key_of(qv), ka = key_of(qa), kb = key_of(qb), kc = key_of(qc);
    unsigned long long km = kv;
    int m = 0;
    if (ka > km) { km = ka; m = 1; }
    if (kb > km) { km = kb; m = 2; }
    if (kc > km) { km = kc; m = 3; }
    long long o;
    switch (m) {
    case 0: o = orient3(a, b, c); break;
    case 1: o = -cross(b, c); break;
    case 2: o = cross(a, c); break;
    default: o = -cross(a, b); break;
    }
    return o > 0 ? 1 : -1;
}

// Apex of the Delaunay triangle to the left of the directed edge v -> w, among the region's
// particles.  Returns its slot, or -1 when there is none or its circumcircle is not certified
// to lie inside the region.
// With a cutoff D (dmax > 0), candidates farther than D from v are skipped, and the result is
// certified only if the circumcircle also lies within distance D of v (its diameter through v
// is at most D), so that no skipped particle can be inside it.
__device__ __forceinline__ int apex_search(const Bins &B, uint2 pv, uint2 pw, const Region &g,
                                           float dmax = 0.f)
{
    const int2 dw = rel(pw, pv);
    const float d2cut = dmax > 0.f ? dmax * dmax : 3.4e38f;
    int best = -1;
    int2 db = make_int2(0, 0);
    uint2 qb = make_uint2(0, 0);
    Circ cb;
    cb.K = cb.P = cb.Q = cb.Pa = cb.Qa = 0.f;
    for_region(B, g, [&](int s) {
        const uint2 qs = __ldg(B.q + s);
        const int2 dc = rel(qs, pv);
        const float fx = (float)dc.x, fy = (float)dc.y;
        if (fmaf(fx, fx, fy * fy) > d2cut) return;    // beyond the cutoff
        if (cross(dw, dc) <= 0) return;               // not strictly left of v -> w
        if (best >= 0) {
            int t = circ_filter(cb, dc);
            if (t == 0) t = incircle_exact(dw, db, dc, pv, pw, qb, qs);
            if (t < 0) return;
        }
        best = s;
        db = dc;
        qb = qs;
        cb = make_circ(dw, dc);
    });
    if (best < 0) return -1;
    // Certify: centre (-P/2K, -Q/2K) relative to v, radius |centre|, plus an error margin far
    // above the FP32 rounding of P, Q, K.
    const float inv2k = 0.5f / cb.K;
    const float cx = -cb.P * inv2k, cy = -cb.Q * inv2k;
    const float r = sqrtf(fmaf(cx, cx, cy * cy));
    const float err = 1e-5f * (cb.Pa + cb.Qa) * (2.f * inv2k) + 64.f;
    const float ext = r + err;
    if (cx - ext < -g.cl_lo_x || cx + ext > g.cl_hi_x || cy - ext < -g.cl_lo_y ||
        cy + ext > g.cl_hi_y)
        return -1;
    if (dmax > 0.f && 2.f * ext > dmax * 0.9999f) return -1;
    return best;
}

// ---------------------------------------------------------------- list-based star (fast path)
// The candidates within distance D of v are gathered once into a per-thread list of FP32
// coordinates relative to v (exact when |d| < 2^24), and the gift-wrap scans run over the
// list with FP32-filtered orientation and incircle tests; a test the filter cannot decide is
// redone exactly from the fixed-point coordinates.  Every returned triangle is certified: its
// circumcircle lies inside the searched region and within distance D of v, so no particle
// left out of the list can be inside it.

#ifndef PFEM_STAR_LIST
#define PFEM_STAR_LIST 24
#endif
constexpr int KL = PFEM_STAR_LIST;   // list capacity (jittered lattices: at most 17 within 2 spacings)

struct FCirc {
    float K, P, Q, Ka, Pa, Qa;
};

__device__ __forceinline__ FCirc make_fcirc(float ax, float ay, float bx, float by)
{
    FCirc c;
    const float la = fmaf(ax, ax, ay * ay), lb = fmaf(bx, bx, by * by);
    const float k1 = ax * by, k2 = ay * bx;
    const float t1 = lb * ay, t2 = la * by, t3 = la * bx, t4 = lb * ax;
    c.K = k1 - k2;  c.Ka = fabsf(k1) + fabsf(k2);
    c.P = t1 - t2;  c.Pa = fabsf(t1) + fabsf(t2);
    c.Q = t3 - t4;  c.Qa = fabsf(t3) + fabsf(t4);
    return c;
}

// +1 inside, -1 outside, 0 undecided.  Inputs carry at most one rounding each; the bound
// (2^-19 of the summed magnitudes, 32 roundings) covers inputs, K/P/Q and the evaluation.
__device__ __forceinline__ int fcirc_filter(const FCirc &c, float x, float y)
{
    const float l = fmaf(x, x, y * y);
    const float det = fmaf(c.K, l, fmaf(c.P, x, c.Q * y));
    const float mag = fmaf(c.Ka, l, fmaf(c.Pa, fabsf(x), c.Qa * fabsf(y)));
    const float bound = 1.9073486328125e-06f * mag;
    return det < -bound ? 1 : (det > bound ? -1 : 0);
}

// Candidate list of the list-based star: thread-private arrays, or a thread's column of a
// shared-memory array (entry k of thread t at k * stride + t).
template <int KLC> struct LocalList {
    float2 xy[KLC];
    int s[KLC];
    __device__ __forceinline__ float2 at(int k) const { return xy[k]; }
    __device__ __forceinline__ int slot(int k) const { return s[k]; }
    __device__ __forceinline__ void put(int k, float2 v, int sl) { xy[k] = v; s[k] = sl; }
};

struct SmemList {
    float2 *xy;
    int *s;
    int stride;
    __device__ __forceinline__ float2 at(int k) const { return xy[k * stride]; }
    __device__ __forceinline__ int slot(int k) const { return s[k * stride]; }
    __device__ __forceinline__ void put(int k, float2 v, int sl) { xy[k * stride] = v; s[k * stride] = sl; }
};

// The star of v from the candidates within distance D of it (list capacity KLC), written as
// out(index, slot) in counter-clockwise order from the nearest neighbour.  Returns the count,
// -1 when the list overflows or a triangle cannot be certified (the caller tries a wider
// search), or -PFEM_ERR_*.
template <int KLC, typename List, typename Out>
static __device__ __forceinline__ int star_list_into(const Bins &B, int v, uint2 pv,
                                                     const Region &g, float D, List &L, Out &&out)
{
    int cnt = 0, u0 = -1, s0 = 0x7fffffff;
    long long d2b = 0x7fffffffffffffffLL;
    bool dup = false, over = false;
    const float D2 = D * D;
    for_region(B, g, [&](int s) {
        if (s == v) return;
        const int2 d = rel(__ldg(B.q + s), pv);
        const float fx = (float)d.x, fy = (float)d.y;
        const float l = fmaf(fx, fx, fy * fy);
        if (l > D2) return;
        const long long d2 = (long long)d.x * d.x + (long long)d.y * d.y;
        dup |= d2 == 0;
        if (cnt == KLC) { over = true; return; }
        L.put(cnt, make_float2(fx, fy), s);
        if (d2 < d2b || (d2 == d2b && s < s0)) { d2b = d2; u0 = cnt; s0 = s; }
        ++cnt;
    });
    if (dup) return -PFEM_ERR_DEGENERATE;
    if (over || u0 < 0) return -1;
    const float clx = g.cl_lo_x, chx = g.cl_hi_x, cly = g.cl_lo_y, chy = g.cl_hi_y;
    int cur = u0, n = 0;
    for (;;) {
        if (n == B.kcap) return -PFEM_ERR_CAPACITY;
        const float2 W = L.at(cur);
        const int wslot = L.slot(cur);
        out(n++, wslot);
        const float wx = W.x, wy = W.y, lw = fmaf(wx, wx, wy * wy);
        int best = -1;
        FCirc cb;
        cb.K = cb.P = cb.Q = cb.Ka = cb.Pa = cb.Qa = 0.f;
        for (int k = 0; k < cnt; ++k) {
            const float2 c2 = L.at(k);
            const float4 c = make_float4(c2.x, c2.y, fmaf(c2.x, c2.x, c2.y * c2.y), 0.f);
            // orientation of (v, w, c): FP32 filter
            const float o1 = wx * c.y, o2 = wy * c.x;
            const float o = o1 - o2;
            const float ob = 4.76837158203125e-07f * (fabsf(o1) + fabsf(o2));
            bool left = o > ob;
            if (fabsf(o) <= ob && k != cur) {            // rare: decide exactly
                const int2 dw = rel(__ldg(B.q + wslot), pv);
                const int2 dc = rel(__ldg(B.q + L.slot(k)), pv);
                left = cross(dw, dc) > 0;
            }
            if (!left) continue;
            if (best >= 0) {
                // inside circle(v, w, best)?  det = K l + P x + Q y < 0
                const float det = fmaf(cb.K, c.z, fmaf(cb.P, c.x, cb.Q * c.y));
                const float mag = fmaf(cb.Ka, c.z, fmaf(cb.Pa, fabsf(c.x), cb.Qa * fabsf(c.y)));
                const float bnd = 1.9073486328125e-06f * mag;
                int t = det < -bnd ? 1 : (det > bnd ? -1 : 0);
                if (t == 0) {                              // rare: decide exactly
                    const uint2 qw = __ldg(B.q + wslot), qb = __ldg(B.q + L.slot(best)),
                                qc = __ldg(B.q + L.slot(k));
                    t = incircle_exact(rel(qw, pv), rel(qb, pv), rel(qc, pv), pv, qw, qb, qc);
                }
                if (t < 0) continue;
            }
            best = k;
            // circle through v, w, c: K = w x c, P = |c|^2 wy - |w|^2 cy, Q = |w|^2 cx - |c|^2 wx
            const float k1 = wx * c.y, k2 = wy * c.x;
            const float t1 = c.z * wy, t2 = lw * c.y, t3 = lw * c.x, t4 = c.z * wx;
            cb.K = k1 - k2;  cb.Ka = fabsf(k1) + fabsf(k2);
            cb.P = t1 - t2;  cb.Pa = fabsf(t1) + fabsf(t2);
            cb.Q = t3 - t4;  cb.Qa = fabsf(t3) + fabsf(t4);
        }
        if (best < 0) return -1;
        // certify: circumcircle centre (-P/2K, -Q/2K), radius |centre|, error margin far above
        // the FP32 rounding of K, P, Q
        const float ak = fabsf(cb.K);
        if (!(ak > 1e-3f * cb.Ka)) return -1;
        const float inv2k = 0.5f / cb.K;
        const float ccx = -cb.P * inv2k, ccy = -cb.Q * inv2k;
        const float r = sqrtf(fmaf(ccx, ccx, ccy * ccy));
        const float err = 1e-4f * (cb.Pa + cb.Qa + (fabsf(cb.P) + fabsf(cb.Q)) * cb.Ka / ak) / ak + 64.f;
        const float ext = r + err;
        if (ccx - ext < -clx || ccx + ext > chx || ccy - ext < -cly || ccy + ext > chy) return -1;
        if (2.f * ext > D * 0.9999f) return -1;
        if (best == u0) break;
        cur = best;
    }
    return n >= 3 ? n : -1;
}

template <int KLC = KL>
static __device__ __forceinline__ int star_list(const Bins &B, int v, uint2 pv, const Region &g,
                                             float D, int *nbrs)
{
    LocalList<KLC> L;
    return star_list_into<KLC>(B, v, pv, g, D, L, [&](int k, int s) { nbrs[k] = s; });
}

// Next search radius: one bin at a time near the first radius, then by a quarter (a large void
// needs few attempts; any radius that certifies a result gives the same, unique result).
__device__ __forceinline__ int next_radius(int R, int R0)
{
    return R < R0 + 3 ? R + 1 : R + max(1, R >> 2);
}

// Star of v by gift-wrapping over every particle of growing regions (no distance cutoff): the
// path of a star the list attempt could not certify.
static __device__ __noinline__ int star_region(const Bins &B, int v, uint2 pv, int R0, int *nbrs)
{
    // First a list attempt with a 1.75 times larger cutoff and a 64-entry list over the bins
    // that cover it (irregular particle sets: on uniform random particles 44 % of the stars
    // have a circumcircle wider than 2 mean spacings, 0.3 % wider than 3.5).
    if (B.dmax > 0.f) {
        const float D2 = B.dmax * 1.75f;
        const float bw = 4294967296.0f / (float)B.nb;
        const int R2 = (int)ceilf(D2 / bw);
        if (R2 <= B.rmax) {
            const int c = star_list<64>(B, v, pv, make_region(B, pv, R2 > R0 ? R2 : R0), D2, nbrs);
            if (c != -1) return c;
        }
    }
    for (int R = R0; R <= B.rmax; R = next_radius(R, R0)) {
        const float dmax = 0.f;
        const Region g = make_region(B, pv, R);
        int u0 = -1;
        long long d2b = 0x7fffffffffffffffLL;
        bool dup = false;
        for_region(B, g, [&](int s) {
            if (s == v) return;
            const int2 d = rel(__ldg(B.q + s), pv);
            const long long d2 = (long long)d.x * d.x + (long long)d.y * d.y;
            dup |= d2 == 0;
            if (d2 < d2b || (d2 == d2b && s < u0)) {
                d2b = d2;
                u0 = s;
            }
        });
        if (dup) return -PFEM_ERR_DEGENERATE;
        if (u0 < 0) continue;
        int cur = u0, cnt = 0;
        bool ok = true;
        for (;;) {
            if (cnt == B.kcap) return -PFEM_ERR_CAPACITY;
            nbrs[cnt++] = cur;
            const int a = apex_search(B, pv, __ldg(B.q + cur), g, dmax);
            if (a < 0) { ok = false; break; }
            if (a == u0) break;
            cur = a;
        }
        if (ok && cnt >= 3) return cnt;
    }
    return -PFEM_FAR;
}

// Counter-clockwise Delaunay star of slot v into nbrs[0..count), starting at v's nearest
// neighbour.  Returns count >= 3, or -PFEM_ERR_* on failure.
static __device__ __noinline__ int star_of(const Bins &B, int v, int R0, int *nbrs)
{
    const uint2 pv = __ldg(B.q + v);
    if (B.dmax > 0.f) {
        const int c = star_list(B, v, pv, make_region(B, pv, R0), B.dmax, nbrs);
        if (c != -1) return c;
    }
    return star_region(B, v, pv, R0, nbrs);
}

// Apex left of the directed edge u -> w, searching around u with growing regions.
__device__ __forceinline__ int apex_of(const Bins &B, int u, int w, int R0)
{
    const uint2 pu = __ldg(B.q + u), pw = __ldg(B.q + w);
    const int a0 = apex_search(B, pu, pw, make_region(B, pu, R0), B.dmax);
    if (a0 >= 0) return a0;
    for (int R = R0; R <= B.rmax; R = next_radius(R, R0)) {
        const int a = apex_search(B, pu, pw, make_region(B, pu, R));
        if (a >= 0) return a;
    }
    return -1;
}

// The particle nearest to fixed-point point p (lowest slot among equals), certified by the
// searched region's clearance; -PFEM_FAR when no region up to rmax certifies it.
__device__ __forceinline__ int nearest_particle(const Bins &B, uint2 p, int R0)
{
    for (int R = R0; R <= B.rmax; R = next_radius(R, R0)) {
        const Region g = make_region(B, p, R);
        long long d2b = 0x7fffffffffffffffLL;
        int best = -1;
        for_region(B, g, [&](int s) {
            const int2 d = rel(__ldg(B.q + s), p);
            const long long d2 = (long long)d.x * d.x + (long long)d.y * d.y;
            if (d2 < d2b || (d2 == d2b && s < best)) {
                d2b = d2;
                best = s;
            }
        });
        const float clm = fminf(fminf(g.cl_lo_x, g.cl_hi_x), fminf(g.cl_lo_y, g.cl_hi_y));
        if (best >= 0 && (float)d2b * 1.0001f < clm * clm) return best;
    }
    return -PFEM_FAR;
}

// The triangle containing p, given the particle v0 nearest to p and its counter-clockwise star
// s0 (cnt entries, any indexable type): the sector of v0's fan that holds p, else a visibility
// walk from that sector's outer edge, stepping through apex(u, w) = the apex of the triangle to
// the left of the directed edge u -> w.  tri = counter-clockwise triangle, with tri[0] = v0 when
// p lies in v0's fan.  Returns 0 or -PFEM_ERR_* / -PFEM_FAR.
template <typename SA, typename Apex>
__device__ __forceinline__ int fan_walk(const Bins &B, uint2 p, int v0, const SA &s0, int cnt,
                                        Apex &&apex, int tri[3])
{
    const uint2 q0 = __ldg(B.q + v0);
    const int2 dp = rel(p, q0);
    if (dp.x == 0 && dp.y == 0) {
        tri[0] = v0; tri[1] = s0[0]; tri[2] = s0[1];
        return 0;
    }
    // sector of the fan around v0 that holds p: [st[j], st[j+1]) counter-clockwise
    int j = -1;
    int2 da = rel(__ldg(B.q + s0[cnt - 1]), q0);
    for (int k = 0; k < cnt; ++k) {
        const int2 dn = rel(__ldg(B.q + s0[k]), q0);
        if (cross(da, dp) >= 0 && cross(dn, dp) < 0) { j = (k + cnt - 1) % cnt; break; }
        da = dn;
    }
    if (j < 0) return -PFEM_ERR_DEGENERATE;
    int e0 = s0[j], e1 = s0[(j + 1) % cnt];
    {
        const int2 a = rel(__ldg(B.q + e0), p), b = rel(__ldg(B.q + e1), p);
        if (cross(a, b) >= 0) {                       // orient(e0, e1, p) >= 0
            tri[0] = v0; tri[1] = e0; tri[2] = e1;
            return 0;
        }
    }
    // visibility walk: p is strictly right of e0 -> e1; step into the triangle beyond.
    for (int step = 0; step < B.walk_cap; ++step) {
        const int x = apex(e1, e0);
        if (x < 0) return x == -1 ? -PFEM_FAR : x;
        const int2 a = rel(__ldg(B.q + e0), p), b = rel(__ldg(B.q + e1), p),
                   c = rel(__ldg(B.q + x), p);
        if (cross(a, c) < 0) { e1 = x; continue; }   // p strictly right of e0 -> x
        if (cross(c, b) < 0) { e0 = x; continue; }   // p strictly right of x -> e1
        tri[0] = e1; tri[1] = e0; tri[2] = x;
        return 0;
    }
    return -PFEM_ERR_TIMEOUT;
}

// Locate fixed-point point p in the Delaunay triangulation: tri = counter-clockwise triangle
// containing p (boundary included).  On success also returns the star of tri[0] in star0
// (count n0) when tri[0] is the particle nearest to p, else n0 = 0.  Returns 0 or -PFEM_ERR_*
// (-PFEM_FAR: a search region reached rmax).
static __device__ __noinline__ int locate(const Bins &B, uint2 p, int R0, int tri[3], int *star0, int &n0)
{
    n0 = 0;
    const int v0 = nearest_particle(B, p, R0);
    if (v0 < 0) return v0;
    const int cnt = star_of(B, v0, R0, star0);
    if (cnt < 0) return cnt;
    const int st = fan_walk(B, p, v0, star0, cnt, [&](int u, int w) { return apex_of(B, u, w, R0); },
                            tri);
    if (st == 0 && tri[0] == v0) n0 = cnt;
    return st;
}

}  // namespace pfem
