// startab.cuh -- the Delaunay star of every particle (App. B: the particles joined to it by a
// Delaunay edge), computed once per projection call and kept in a table that the per-node
// kernels read instead of searching.
//
// A mesh node needs the stars of the three vertices of its Delaunay triangle, and neighbouring
// nodes need different particles; searching stars per node makes every thread of a warp run its
// own gift-wrapping, of its own length, over its own candidate list.  Here every particle's star
// is computed by one thread of a particle-parallel kernel, so the threads of a warp do the same
// work on neighbouring particles (consecutive slots share bins), with the candidate lists in
// shared memory.  Stars the list attempt cannot certify (an empty circle wider than the
// candidate cutoff, a list overflow) are queued and computed by a second kernel that searches
// growing regions.  The table is then a plain array: slot v's star is nbr[v * PFEM_KMAX + k],
// k < cnt[v], counter-clockwise from its nearest neighbour.
#pragma once

#include "geom.cuh"

namespace pfem {

struct StarTab {
    int *nbr;           // [N][KMAX] slots
    int *cnt;           // [N] star size (>= 3), -1 while queued, or -PFEM_ERR_*
    int *queue;         // [N] slots whose list attempt failed
    int *qcount;        // number of queued slots
    long long N;
};

// Star of slot v read from the table (entries through the read-only cache).
struct TabStar {
    const int *p;
    int n;
    __device__ __forceinline__ int operator[](int i) const { return __ldg(p + i); }
};

__device__ __forceinline__ TabStar tab_star(const StarTab &t, int v)
{
    return {t.nbr + (long long)v * KMAX, __ldg(t.cnt + v)};
}

// Apex of the Delaunay triangle to the left of the directed edge u -> w: the neighbour that
// follows w counter-clockwise in u's star.  -PFEM_ERR_DEGENERATE if w is not in u's star (the
// table is then inconsistent, which exact predicates rule out), or u's star's error.
__device__ __forceinline__ int tab_apex(const StarTab &t, int u, int w)
{
    const TabStar s = tab_star(t, u);
    if (s.n < 0) return s.n;
    for (int k = 0; k < s.n; ++k)
        if (s[k] == w) return s[k + 1 == s.n ? 0 : k + 1];
    return -PFEM_ERR_DEGENERATE;
}

// Locate fixed-point point p with the table's stars: nearest particle, the sector of its fan,
// else a visibility walk whose steps are table lookups.  Returns 0 or -PFEM_ERR_* / -PFEM_FAR.
static __device__ __noinline__ int locate_tab(const Bins &B, const StarTab &t, uint2 p, int R0,
                                              int tri[3])
{
    const int v0 = nearest_particle(B, p, R0);
    if (v0 < 0) return v0;
    const TabStar s0 = tab_star(t, v0);
    if (s0.n < 0) return s0.n;
    return fan_walk(B, p, v0, s0, s0.n, [&](int u, int w) { return tab_apex(t, u, w); }, tri);
}

// Threads per block and candidate-list capacity of the list kernels.  The lists live in shared
// memory, one column per thread (18 candidates x 17 bytes x 128 threads = 39 KB per block).
// Jittered lattices have at most 17 particles within the 2-spacing cutoff; longer lists go to the
// retry kernel.
constexpr int STAR_TPB = 128;
#ifndef PFEM_STAR_KL
#define PFEM_STAR_KL 18
#endif
constexpr int STAR_KL = PFEM_STAR_KL;

// A thread's candidate list for the hull star: coordinates relative to v (FP32), angular key
// and slot per candidate, the candidates' order by angle (list indices), and the hull stack
// (list indices); entry k of thread t at k * stride + t.
struct HullList {
    float2 *xy;
    float *key;
    int *s;
    unsigned char *ord;
    unsigned char *stk;
    int stride;
};

// Pseudo-angle of (x, y) in [0, 4): monotone in the polar angle (0 along +x, 1 along +y, ...);
// the quadrant is decided by the signs of x and y, so the ends of the range never mix.
__device__ __forceinline__ float pseudo_angle(float x, float y)
{
    const float p = __fdividef(y, fabsf(x) + fabsf(y));
    return x >= 0.f ? (y >= 0.f ? p : 4.f + p) : 2.f - p;
}

// Keys closer than this may be out of order after FP32 rounding (their error is below 1e-6):
// such pairs are ordered exactly.
constexpr float KEY_EPS = 4e-6f;

// The Delaunay star of v from the candidates within distance D (capacity KLC), by the convex
// hull of the candidates inverted about v.  Inversion c -> c/|c|^2 maps the circles through v
// to lines, so an empty circle through v, a, b becomes a hull edge between the images of a
// and b; and the orientation of three images is the sign of the lifted incircle determinant of
// (v, a, b, c) -- the predicate of the gift-wrapping search, with the same tie-break.  So the
// hull's vertices in counter-clockwise order are v's star.  Steps: gather the candidates (the
// nearest one, u0, is always a Delaunay neighbour), order them by angle about v, one Graham
// scan starting at u0, then certify every triangle (v, w_j, w_j+1) as the gift-wrapping search
// does (the circumcircle inside the searched region and within D of v).  Returns the count,
// -1 (list overflow or not certified: the caller retries wider) or -PFEM_ERR_*.
template <int KLC, typename Out>
__device__ __forceinline__ int star_hull(const Bins &B, int v, uint2 pv, const Region &g, float D,
                                         const HullList &L, Out &&out)
{
    const int S = L.stride;
    int cnt = 0, u0 = -1, s0 = 0x7fffffff;
    long long d2b = 0x7fffffffffffffffLL;
    float lb = 3.4e38f;
    bool dup = false, over = false;
    const float D2 = D * D;
    for_region(B, g, [&](int s) {
        if (s == v) return;
        const int2 d = rel(__ldg(B.q + s), pv);
        const float fx = (float)d.x, fy = (float)d.y;
        const float l = fmaf(fx, fx, fy * fy);
        if (l > D2) return;
        dup |= (d.x | d.y) == 0;
        if (cnt == KLC) { over = true; return; }
        L.xy[cnt * S] = make_float2(fx, fy);
        L.key[cnt * S] = pseudo_angle(fx, fy);
        L.s[cnt * S] = s;
        if (l <= lb * 1.000001f) {             // near the nearest so far: decide exactly
            const long long d2 = (long long)d.x * d.x + (long long)d.y * d.y;
            if (d2 < d2b || (d2 == d2b && s < s0)) { d2b = d2; u0 = cnt; s0 = s; lb = l; }
        }
        ++cnt;
    });
    if (dup) return -PFEM_ERR_DEGENERATE;
    if (over || u0 < 0) return -1;
    auto exact_of = [&](int k) { return rel(__ldg(B.q + L.s[k * S]), pv); };
    // Order by angle (insertion sort of indices).  Should candidate a come after b?  Near-equal
    // keys are ordered by the exact cross product, and on one ray the farther particle comes
    // first: its image lies inside the hull and the scan removes it; on u0's ray this puts
    // the farther particles just before u0, i.e. at the end of the scan that starts at u0.
    auto after = [&](int a, float ka, int b, float kb) -> bool {
        if (ka - kb > KEY_EPS) return true;
        if (kb - ka > KEY_EPS) return false;
        const int2 da = exact_of(a), db = exact_of(b);
        const long long cr = cross(da, db);
        if (cr != 0) return cr < 0;
        return (long long)da.x * da.x + (long long)da.y * da.y <
               (long long)db.x * db.x + (long long)db.y * db.y;
    };
    L.ord[0] = 0;
    for (int i = 1; i < cnt; ++i) {
        const float ki = L.key[i * S];
        int j = i - 1;
        for (; j >= 0; --j) {
            const int oj = L.ord[j * S];
            if (!after(oj, L.key[oj * S], i, ki)) break;
            L.ord[(j + 1) * S] = (unsigned char)oj;
        }
        L.ord[(j + 1) * S] = (unsigned char)i;
    }
    int p0 = 0;
    for (int i = 0; i < cnt; ++i)
        if (L.ord[i * S] == u0) p0 = i;
    // Graham scan, cyclically from u0.  left(a, b, c): is the image of c to the left of the
    // images of a -> b, i.e. c outside the circle through v, a, b?  FP32 filter on
    // det = la (b x c) - lb (a x c) + lc (a x b), whose terms are bounded by
    // la lb + lc (la + lb) (|p x q| <= (lp + lq) / 2); the exact predicate when undecided.
    auto left = [&](int a, int b, int c) -> bool {
        const float2 A = L.xy[a * S], Bp = L.xy[b * S], Cp = L.xy[c * S];
        const float la = fmaf(A.x, A.x, A.y * A.y), lbb = fmaf(Bp.x, Bp.x, Bp.y * Bp.y),
                    lc = fmaf(Cp.x, Cp.x, Cp.y * Cp.y);
        const float bc = fmaf(Bp.x, Cp.y, -Bp.y * Cp.x), ac = fmaf(A.x, Cp.y, -A.y * Cp.x),
                    ab = fmaf(A.x, Bp.y, -A.y * Bp.x);
        const float det = fmaf(la, bc, fmaf(-lbb, ac, lc * ab));
        const float bnd = 1.9073486328125e-06f * fmaf(la, lbb, lc * (la + lbb));
        if (det > bnd) return true;
        if (det < -bnd) return false;
        const uint2 qa = __ldg(B.q + L.s[a * S]), qb = __ldg(B.q + L.s[b * S]),
                    qc = __ldg(B.q + L.s[c * S]);
        return incircle_exact(rel(qa, pv), rel(qb, pv), rel(qc, pv), pv, qa, qb, qc) < 0;
    };
    L.stk[0] = (unsigned char)u0;
    int sp = 1;
    for (int i = 1, p = p0 + 1; i < cnt; ++i, ++p) {
        const int c = L.ord[(p == cnt ? (p = 0) : p) * S];
        while (sp >= 2 && !left(L.stk[(sp - 2) * S], L.stk[(sp - 1) * S], c)) --sp;
        L.stk[sp * S] = (unsigned char)c;
        ++sp;
    }
    while (sp >= 3 && !left(L.stk[(sp - 2) * S], L.stk[(sp - 1) * S], u0)) --sp;
    if (sp < 3) return -1;
    // certify every triangle (v, w_j, w_j+1): counter-clockwise, circumcircle inside the region
    // and within D of v (then no particle outside the list can lie inside it).  The circle
    // through v, a, b has centre -(P, Q) / 2K and passes through v; its radius r must satisfy
    // r + err <= every clearance measured from the centre and <= D / 2.
    for (int j = 0; j < sp; ++j) {
        const float2 a = L.xy[L.stk[j * S] * S];
        const float2 b = L.xy[L.stk[(j + 1 == sp ? 0 : j + 1) * S] * S];
        const FCirc cb = make_fcirc(a.x, a.y, b.x, b.y);
        if (!(cb.K > 1e-3f * cb.Ka)) return -1;
        const float ik = __frcp_rn(cb.K);
        const float ccx = -0.5f * cb.P * ik, ccy = -0.5f * cb.Q * ik;
        const float err = (1e-4f * (cb.Pa + cb.Qa + (fabsf(cb.P) + fabsf(cb.Q)) * cb.Ka * ik)) * ik + 64.f;
        const float room = fminf(fminf(fminf(g.cl_hi_x - ccx, g.cl_lo_x + ccx),
                                       fminf(g.cl_hi_y - ccy, g.cl_lo_y + ccy)),
                                 0.49995f * D) - err;
        if (!(room > 0.f) || fmaf(ccx, ccx, ccy * ccy) > room * room * 0.9999f) return -1;
    }
    if (sp > B.kcap) return -PFEM_ERR_CAPACITY;
    for (int j = 0; j < sp; ++j) out(j, L.s[L.stk[j * S] * S]);
    return sp;
}

// The list attempt for slot v (candidates in L): its star into the table, or v queued.
__device__ __forceinline__ void star_list_slot(const Bins &B, int R0, const StarTab &t, long long v,
                                               const HullList &L, DevStatus *st)
{
    const uint2 pv = __ldg(B.q + v);
    int *out = t.nbr + v * KMAX;
    int c = -1;
    if (B.dmax > 0.f)
        c = star_hull<STAR_KL>(B, (int)v, pv, make_region(B, pv, R0), B.dmax, L,
                               [&](int k, int s) { out[k] = s; });
    if (c == -1) {
        t.cnt[v] = -1;
        t.queue[atomicAdd(t.qcount, 1)] = (int)v;   // at most N entries: each slot once
        return;
    }
    t.cnt[v] = c;
    if (c < 0) record_error(st, -c, v);
}

// A queued slot: the wide list attempt and then growing regions (star_region) up to B.rmax.  A
// star that still fails records its error (an exhausted region as PFEM_ERR_CAPACITY).
__device__ __forceinline__ void star_retry_slot(const Bins &B, int R0, const StarTab &t, int v,
                                                DevStatus *st)
{
    int loc[KMAX];
    int c = star_region(B, v, __ldg(B.q + v), R0, loc);
    if (c > 0) {
        int *out = t.nbr + (long long)v * KMAX;
        for (int k = 0; k < c; ++k) out[k] = loc[k];
    } else {
        if (c == -PFEM_FAR || c == -1) c = -PFEM_ERR_CAPACITY;
        record_error(st, -c, v);
    }
    t.cnt[v] = c;
}

}  // namespace pfem
