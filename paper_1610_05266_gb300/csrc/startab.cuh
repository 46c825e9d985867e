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

// Threads per block and candidate-list capacity of the list kernels.  The list lives in shared
// memory, one column per thread (20 x 12 bytes x 128 threads = 30 KB per block, 7 blocks per SM).
// Jittered lattices have at most 17 particles within the 2-spacing cutoff; longer lists go to the
// retry kernel.
constexpr int STAR_TPB = 128;
#ifndef PFEM_STAR_KL
#define PFEM_STAR_KL 20
#endif
constexpr int STAR_KL = PFEM_STAR_KL;

// The list attempt for slot v (candidates in L): its star into the table, or v queued.
__device__ __forceinline__ void star_list_slot(const Bins &B, int R0, const StarTab &t, long long v,
                                               SmemList &L, DevStatus *st)
{
    const uint2 pv = __ldg(B.q + v);
    int *out = t.nbr + v * KMAX;
    int c = -1;
    if (B.dmax > 0.f)
        c = star_list_into<STAR_KL>(B, (int)v, pv, make_region(B, pv, R0), B.dmax, L,
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
