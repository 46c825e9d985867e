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
    int *cnt;           // [N] stamped count (tab_pack): star size, -1 while queued, or -PFEM_ERR_*
    int *queue;         // [N] slots whose list attempt failed
    int *qcount;        // number of queued slots
    long long N;
    unsigned gen;       // stamp of this call's entries (1 .. 2^24 - 1)
};

// A count entry carries the stamp of the call that wrote it, so that an entry left by an
// earlier call (or not yet written by this one) reads as "not available" (-1) instead of as a
// star: (gen << 8) | (value + 128).
__device__ __forceinline__ int tab_pack(unsigned gen, int v)
{
    return (int)((gen << 8) | (unsigned)((v + 128) & 255));
}

__device__ __forceinline__ int tab_count(const StarTab &t, int v)
{
    const unsigned w = (unsigned)__ldg(t.cnt + v);
    return (w >> 8) == t.gen ? (int)(w & 255u) - 128 : -1;
}

// Star of slot v read from the table (entries through the read-only cache).
struct TabStar {
    const int *p;
    int n;
    __device__ __forceinline__ int operator[](int i) const { return __ldg(p + i); }
};

__device__ __forceinline__ TabStar tab_star(const StarTab &t, int v)
{
    return {t.nbr + (long long)v * KMAX, tab_count(t, v)};
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
    if (s0.n < 0) return s0.n == -1 ? -PFEM_FAR : s0.n;
    return fan_walk(B, p, v0, s0, s0.n, [&](int u, int w) { return tab_apex(t, u, w); }, tri);
}

// Threads per block and candidate-list capacity of the list kernels.  The lists live in shared
// memory, one column per thread (16 candidates x 18 bytes x 128 threads = 36 KB per block).
// Jittered lattices at jitter 0.25 have at most 16 particles within the 2-spacing cutoff (rarely
// 17 at jitter 0.3); longer lists go to the retry kernel.
constexpr int STAR_TPB = 128;
constexpr int STAR_KL = 16;

// A thread's candidate list for the hull star: coordinates relative to v (FP32), the packed
// angular key, the slot, the order by angle and the hull stack; entry k of thread t at
// k * stride + t.
struct HullList {
    float2 *xy;
    unsigned *pk;
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

// The key of candidate k, packed for sorting: the pseudo-angle in 27-bit fixed point (units of
// 2^-25) above the 5-bit list index.  The pseudo-angle's FP32 error is below 1e-6, so keys that
// differ by more than KEY_NEAR units are in the right order; closer ones are ordered exactly.
constexpr unsigned KEY_NEAR = 134;   // 4e-6 * 2^25
__device__ __forceinline__ unsigned pack_key(float x, float y, int k)
{
    const float a = fminf(pseudo_angle(x, y), 3.9999998f);
    return ((unsigned)(a * 33554432.0f) << 5) | (unsigned)k;
}

// Sort KLC packed keys (bitonic network, unrolled: the array stays in registers; Batcher's
// odd-even merge network, 63 instead of 80 compare-exchanges for 16 keys, measured slower).
template <int KLC> __device__ __forceinline__ void sort_keys(unsigned (&w)[KLC])
{
#pragma unroll
    for (int size = 2; size <= KLC; size <<= 1)
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
            for (int i = 0; i < KLC; ++i) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned a = w[i], b = w[j];
                    const unsigned lo = min(a, b), hi = max(a, b);
                    const bool up = (i & size) == 0;
                    w[i] = up ? lo : hi;
                    w[j] = up ? hi : lo;
                }
            }
}

// The Delaunay star of v from the candidates within distance D (at most KLC, 16 or 32), by the convex
// hull of the candidates inverted about v.  Inversion c -> c/|c|^2 maps the circles through v
// to lines, so an empty circle through v, a, b becomes a hull edge between the images of a
// and b; and the orientation of three images is the sign of the lifted incircle determinant of
// (v, a, b, c) -- the predicate of the gift-wrapping search, with the same tie-break.  So the
// hull's vertices in counter-clockwise order are v's star.  Steps: gather the candidates (the
// nearest one, u0, is always a Delaunay neighbour), order them by angle about v, one Graham
// scan starting at u0, then certify every triangle (v, w_j, w_j+1) as the gift-wrapping search
// does (the circumcircle inside the searched region and within D of v).  Returns the count,
// -1 (list overflow or not certified: the caller retries wider) or -PFEM_ERR_*.
template <int KLC>
__device__ __forceinline__ int star_hull(const Bins &B, int v, uint2 pv, const Region &g, float D,
                                         const HullList &L, int *row)
{
    static_assert(KLC == 16 || KLC == 32, "the packed key holds a 5-bit list index");
    const int S = L.stride;
    int cnt = 0, u0 = -1, s0 = 0x7fffffff;
    long long d2b = 0x7fffffffffffffffLL;
    float lb = 3.4e38f;
    bool dup = false, over = false;
    const float D2 = D * D;
    auto take = [&](int s, uint2 qs) {
        if (s == v) return;
        const int2 d = rel(qs, pv);
        const float fx = (float)d.x, fy = (float)d.y;
        const float l = fmaf(fx, fx, fy * fy);
        if (l > D2) return;
        dup |= (d.x | d.y) == 0;
        if (cnt == KLC) { over = true; return; }
        L.xy[cnt * S] = make_float2(fx, fy);
        L.pk[cnt * S] = pack_key(fx, fy, cnt);
        L.s[cnt * S] = s;
        if (l <= lb * 1.000001f) {             // near the nearest so far: decide exactly
            const long long d2 = (long long)d.x * d.x + (long long)d.y * d.y;
            if (d2 < d2b || (d2 == d2b && s < s0)) { d2b = d2; u0 = cnt; s0 = s; lb = l; }
        }
        ++cnt;
    };
    // the region's slot runs, four loads in flight at a time
    for_region_runs(B, g, [&](int a, int e) {
        int s = a;
        for (; s + 4 <= e; s += 4) {
            const uint2 q0 = __ldg(B.q + s), q1 = __ldg(B.q + s + 1), q2 = __ldg(B.q + s + 2),
                        q3 = __ldg(B.q + s + 3);
            take(s, q0);
            take(s + 1, q1);
            take(s + 2, q2);
            take(s + 3, q3);
        }
        for (; s < e; ++s) take(s, __ldg(B.q + s));
    });
    if (dup) return -PFEM_ERR_DEGENERATE;
    if (over || u0 < 0) return -1;
    auto exact_of = [&](int k) { return rel(__ldg(B.q + L.s[k * S]), pv); };
    // Order by angle: the packed keys through the network, then an exact pass over keys closer
    // than KEY_NEAR (near-equal angles by the exact cross product; on one ray the farther
    // particle first: its image lies inside the hull and the scan removes it, and on u0's ray
    // this puts the farther particles just before u0, i.e. at the end of the scan from u0).
    unsigned w[KLC];
#pragma unroll
    for (int k = 0; k < KLC; ++k) w[k] = k < cnt ? L.pk[k * S] : 0xffffffffu;
    sort_keys<KLC>(w);
    bool near = false;
    int p0 = 0;
#pragma unroll
    for (int k = 0; k < KLC; ++k) {
        if (k < cnt) L.ord[k * S] = (unsigned char)(w[k] & 31u);
        if (k + 1 < cnt && (w[k + 1] >> 5) - (w[k] >> 5) < KEY_NEAR) near = true;
        if (k < cnt && (int)(w[k] & 31u) == u0) p0 = k;
    }
    if (near) {
        auto after = [&](int a, int b) -> bool {   // should candidate a come after b?
            const unsigned ka = L.pk[a * S] >> 5, kb = L.pk[b * S] >> 5;
            if (ka > kb + KEY_NEAR) return true;
            if (kb > ka + KEY_NEAR) return false;
            const int2 da = exact_of(a), db = exact_of(b);
            const long long cr = cross(da, db);
            if (cr != 0) return cr < 0;
            return (long long)da.x * da.x + (long long)da.y * da.y <
                   (long long)db.x * db.x + (long long)db.y * db.y;
        };
        for (int i = 1; i < cnt; ++i) {
            const int oi = L.ord[i * S];
            int j = i - 1;
            for (; j >= 0; --j) {
                const int oj = L.ord[j * S];
                if (!after(oj, oi)) break;
                L.ord[(j + 1) * S] = (unsigned char)oj;
            }
            L.ord[(j + 1) * S] = (unsigned char)oi;
        }
        for (int k = 0; k < cnt; ++k)
            if (L.ord[k * S] == u0) p0 = k;
    }
    // Graham scan, cyclically from u0.  Is the image of c to the left of the images of a -> b,
    // i.e. c outside the circle through v, a, b?  FP32 filter on
    // det = la (b x c) - lb (a x c) + lc (a x b), whose terms are bounded by
    // la lb + lc (la + lb) <= 3 D^4 (|p x q| <= (lp + lq) / 2, every l <= D^2): one bound for the
    // whole star, 2^-19 of that; the exact predicate when undecided.
    // The two top entries of the stack are kept in registers.
    auto xyl = [&](int k, float &x, float &y, float &l) {
        const float2 t = L.xy[k * S];
        x = t.x;
        y = t.y;
        l = fmaf(x, x, y * y);
    };
    int ia = -1, ib = u0;
    float ax = 0.f, ay = 0.f, la = 0.f, bx, by, lbv;
    xyl(u0, bx, by, lbv);
    float ab = 0.f;
    L.stk[0] = (unsigned char)u0;
    int sp = 1;
    const float bnd = 5.7220458984375e-06f * D2 * D2;    // 3 x 2^-19 x D^4
    auto left = [&](int c, float cx, float cy, float lc) -> bool {
        const float bc = fmaf(bx, cy, -by * cx), ac = fmaf(ax, cy, -ay * cx);
        const float det = fmaf(la, bc, fmaf(-lbv, ac, lc * ab));
        if (det > bnd) return true;
        if (det < -bnd) return false;
        const uint2 qa = __ldg(B.q + L.s[ia * S]), qb = __ldg(B.q + L.s[ib * S]),
                    qc = __ldg(B.q + L.s[c * S]);
        return incircle_exact(rel(qa, pv), rel(qb, pv), rel(qc, pv), pv, qa, qb, qc) < 0;
    };
    auto pop = [&]() {
        --sp;
        ib = ia;
        bx = ax;
        by = ay;
        lbv = la;
        if (sp >= 2) {
            ia = L.stk[(sp - 2) * S];
            xyl(ia, ax, ay, la);
            ab = fmaf(ax, by, -ay * bx);
        }
    };
    for (int i = 1, p = p0 + 1; i < cnt; ++i, ++p) {
        if (p == cnt) p = 0;
        const int c = L.ord[p * S];
        float cx, cy, lc;
        xyl(c, cx, cy, lc);
        while (sp >= 2 && !left(c, cx, cy, lc)) pop();
        L.stk[sp * S] = (unsigned char)c;
        ++sp;
        ia = ib; ax = bx; ay = by; la = lbv;
        ib = c; bx = cx; by = cy; lbv = lc;
        ab = fmaf(ax, by, -ay * bx);
    }
    {
        float cx, cy, lc;
        xyl(u0, cx, cy, lc);
        while (sp >= 3 && !left(u0, cx, cy, lc)) pop();
    }
    if (sp < 3) return -1;
    // certify every triangle (v, w_j, w_j+1): counter-clockwise, circumcircle inside the region
    // and within D of v (then no particle outside the list can lie inside it).
    if (fminf(fminf(g.cl_lo_x, g.cl_hi_x), fminf(g.cl_lo_y, g.cl_hi_y)) >= 0.9995f * D) {
        // The region holds the disk of radius 0.9995 D about v.  A circle through v of radius
        // r = |a| |b| |a - b| / (2 |a x b|) lies within 2r of v, so 4 r^2 <= 0.997 D^2, i.e.
        // la lb |a - b|^2 <= 0.997 D^2 K^2, keeps it inside both.  Each FP32 offset carries
        // at most one rounding (2^-24, none below 2^24 units).  With K > 1e-3 of its summed
        // magnitudes, K^2 is within 4e-4 of its exact value, and a and b are then at least
        // 7e-4 rad apart as seen from v, so |a - b|^2 is within 4e-4 as well: the true 2r stays
        // below 0.9989 D, inside the region, and every particle within the circle has an FP32
        // squared distance below D^2, i.e. is in the list.
        const float iD2 = __frcp_rn(D2);
        for (int j = 0; j < sp; ++j) {
            const float2 a = L.xy[L.stk[j * S] * S];
            const float2 b = L.xy[L.stk[(j + 1 == sp ? 0 : j + 1) * S] * S];
            const float k1 = a.x * b.y, k2 = a.y * b.x;
            const float K = k1 - k2;
            if (!(K > 1e-3f * (fabsf(k1) + fabsf(k2)))) {
                // a thin triangle at v: the same bound from the exact offsets (64-bit
                // integers, products in FP64 within 1e-15)
                const int2 ea = exact_of(L.stk[j * S]);
                const int2 eb = exact_of(L.stk[(j + 1 == sp ? 0 : j + 1) * S]);
                const long long Ke = (long long)ea.x * eb.y - (long long)ea.y * eb.x;
                if (Ke <= 0) return -1;
                const long long ex = (long long)ea.x - eb.x, ey = (long long)ea.y - eb.y;
                const double lae = (double)((long long)ea.x * ea.x + (long long)ea.y * ea.y);
                const double lbe = (double)((long long)eb.x * eb.x + (long long)eb.y * eb.y);
                const double labe = ((double)(ex * ex) + (double)(ey * ey)) / ((double)D * (double)D);
                const double Kd = (double)Ke;
                if (lae * lbe * labe > 0.997 * Kd * Kd) return -1;
                continue;
            }
            const float dx = a.x - b.x, dy = a.y - b.y;
            const float la = fmaf(a.x, a.x, a.y * a.y), lb = fmaf(b.x, b.x, b.y * b.y);
            const float lab = fmaf(dx, dx, dy * dy) * iD2;
            if (la * lb * lab > 0.997f * K * K) return -1;
        }
    } else {
    // The circle through v, a, b has centre -(P, Q) / 2K and passes through v; its radius r
    // must satisfy r + err <= every clearance measured from the centre and <= D / 2.
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
    }
    if (sp > B.kcap) return -PFEM_ERR_CAPACITY;
    // the row (64-byte aligned) in whole 32-byte sectors by 16-byte stores, -1 after the star:
    // a partly written sector would cost the memory system a read to complete it
    const int nq = ((sp + 7) >> 3) << 1;
    for (int q = 0; q < nq; ++q) {
        int e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            e[i] = -1;
            if (4 * q + i < sp) e[i] = L.s[L.stk[(4 * q + i) * S] * S];
        }
        reinterpret_cast<int4 *>(row)[q] = make_int4(e[0], e[1], e[2], e[3]);
    }
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
        c = star_hull<STAR_KL>(B, (int)v, pv, make_region(B, pv, R0), B.dmax, L, out);
    if (c == -1) {
        t.cnt[v] = tab_pack(t.gen, -1);
        t.queue[atomicAdd(t.qcount, 1)] = (int)v;   // at most N entries: each slot once
        return;
    }
    t.cnt[v] = tab_pack(t.gen, c);
    if (c < 0) record_error(st, -c, v);
}

// A queued slot, first pass (short queues only): the hull attempt again over a 32-entry list at
// 1.25 times the cutoff (a circumcircle a little wider than the first cutoff: at jitter 0.25 the
// Delaunay circumdiameter of a jittered lattice can reach 2.12 spacings).  A star it cannot
// certify keeps its queued mark for star_retry_slot.
constexpr int STAR_KL_RETRY = 32;
__device__ __forceinline__ void star_retry_hull_slot(const Bins &B, int R0, const StarTab &t, int v,
                                                     const HullList &L, DevStatus *st)
{
    if (!(B.dmax > 0.f)) return;
    const uint2 pv = __ldg(B.q + v);
    int *out = t.nbr + (long long)v * KMAX;
    const float D = 1.25f * B.dmax;
    const int R = max(R0, (int)ceilf(D * (float)B.nb * 2.3283064365386963e-10f));
    if (R > B.rmax) return;
    const int c = star_hull<STAR_KL_RETRY>(B, v, pv, make_region(B, pv, R), D, L, out);
    if (c == -1) return;
    t.cnt[v] = tab_pack(t.gen, c);
    if (c < 0) record_error(st, -c, v);
}

// A queued slot still marked queued: the wide list attempt and then growing regions
// (star_region) up to B.rmax.  A star that still fails records its error (an exhausted region
// as PFEM_ERR_CAPACITY).
__device__ __forceinline__ void star_retry_slot(const Bins &B, int R0, const StarTab &t, int v,
                                                DevStatus *st)
{
    if (tab_count(t, v) != -1) return;
    int loc[KMAX];
    int c = star_region(B, v, __ldg(B.q + v), R0, loc);
    if (c > 0) {
        int *out = t.nbr + (long long)v * KMAX;
        for (int k = 0; k < ((c + 7) & ~7); ++k) out[k] = k < c ? loc[k] : -1;
    } else {
        if (c == -PFEM_FAR || c == -1) c = -PFEM_ERR_CAPACITY;
        record_error(st, -c, v);
    }
    t.cnt[v] = tab_pack(t.gen, c);
}

// Blocks per SM of the region-search retry kernels (64 threads, 96 registers: 10 fit).  The
// queue length is known only on the device, so the grid covers what the SMs hold at once; on
// 2048^2 uniform random particles (2.35M stars queued) 4, 10, 16 blocks measured 11.0, 6.8,
// 7.7 ms, on the jittered lattice (12 queued) no difference.
#ifndef PFEM_RETRY_REGION_BLOCKS
#define PFEM_RETRY_REGION_BLOCKS 10
#endif
// Blocks per SM of the hull retry kernels (64 threads and 36 KB of lists each).
#ifndef PFEM_RETRY_BLOCKS
#define PFEM_RETRY_BLOCKS 6
#endif
// The hull retry runs for queues up to 1/64 of the particles: on irregular particle sets
// (uniform random: 56 % of the stars queued) a quarter of the queued stars fail it too, and the
// wide attempt alone measured faster.
__device__ __forceinline__ bool short_queue(int n, long long N) { return n <= (N >> 6); }

}  // namespace pfem
