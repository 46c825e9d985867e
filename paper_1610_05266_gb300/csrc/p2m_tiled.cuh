// p2m_tiled.cuh -- CTA-tiled particle-to-mesh projection (Sec. 2.2 eq. p2m with the shape
// functions of App. B), the fast path of the fused P2M.
//
// A block owns a T x T tile of mesh nodes.  It stages the fixed-point coordinates of every
// particle in the bins around the tile (a halo of THB bins) in shared memory, relative to the
// tile origin, and then:
//   1. each node finds its nearest particle v0 among the staged particles;
//   2. the stars of all distinct v0 are computed once each (a shared work list), by
//      gift-wrapping over shared-memory candidates, and certified against the searched region;
//   3. each node locates its Delaunay triangle from v0's star (fan sector test, else a
//      visibility walk with apex searches in shared memory);
//   4. the stars of all distinct triangle vertices not yet known are computed once each;
//   5. each node solves its three edge systems (App. B eqs. A0, A1, condquad, minimum norm)
//      and applies the weights to all C components.
// A node whose geometry cannot be certified inside the staged window (or whose tile does not
// fit the staging capacity) takes the per-thread global-memory path instead, which grows its
// search regions as needed; both paths compute the same exact topology.
#pragma once

#include "p2m.cuh"

namespace pfem {

constexpr int TT = 256;        // threads per tile block
constexpr int TMAXP = 3072;    // staged particles per tile
constexpr int TMAXB = 1024;    // staged bins per tile
constexpr int TMAXS = 768;     // stars per tile
constexpr int THB = 3;         // halo bins on each side of the tile's node bins

struct TileSmem {
    int2 rq[TMAXP];                      // fixed point relative to the tile origin
    int gslot[TMAXP];                    // global slot of each staged particle
    unsigned short bstart[TMAXB + 1];    // staged index of each local bin (row-major)
    unsigned short star[TMAXS][KMAX];    // stars, as staged indices
    signed char scount[TMAXS];           // star size, or -(pfem error)
    short sslot[TMAXP];                  // star index per particle: -1 none, -2 claimed
    int work[TMAXS];
    int nwork, np, bad;
    int wbx, wby, bx0, by0;              // window: local bins and its first (unwrapped) bin
    long long Xo, Yo;                    // tile origin, unwrapped fixed point
    uint2 org;                           // tile origin, fixed point
    int scan[TT / 32];
};

// ceil(b * 2^32 / nb) for any integer bin index b (unwrapped)
__device__ __forceinline__ long long blo_u(long long b, int nb)
{
    if (b >= 0) return ((b << 32) + nb - 1) / nb;
    return -(((-b) << 32) / nb);
}

// unwrapped bin of an unwrapped fixed-point coordinate
__device__ __forceinline__ long long bin_u(long long X, int nb) { return (X * nb) >> 32; }

struct SRegion {
    int lx0, lx1, ly0, ly1;
    float cl_lo_x, cl_hi_x, cl_lo_y, cl_hi_y;
};

// Region of +-R bins around staged point p (tile-relative), if it lies inside the window.
__device__ __forceinline__ bool sregion(const TileSmem &S, int nb, int2 p, int R, SRegion &g)
{
    const long long X = S.Xo + p.x, Y = S.Yo + p.y;
    const long long gbx = bin_u(X, nb), gby = bin_u(Y, nb);
    const int lx = (int)(gbx - S.bx0), ly = (int)(gby - S.by0);
    g.lx0 = lx - R; g.lx1 = lx + R; g.ly0 = ly - R; g.ly1 = ly + R;
    if (g.lx0 < 0 || g.ly0 < 0 || g.lx1 >= S.wbx || g.ly1 >= S.wby) return false;
    g.cl_lo_x = (float)(X - blo_u(gbx - R, nb));
    g.cl_hi_x = (float)(blo_u(gbx + R + 1, nb) - 1 - X);
    g.cl_lo_y = (float)(Y - blo_u(gby - R, nb));
    g.cl_hi_y = (float)(blo_u(gby + R + 1, nb) - 1 - Y);
    return true;
}

template <typename F>
__device__ __forceinline__ void for_sregion(const TileSmem &S, const SRegion &g, F &&f)
{
    for (int ly = g.ly0; ly <= g.ly1; ++ly) {
        const int row = ly * S.wbx;
        const int e = S.bstart[row + g.lx1 + 1];
        for (int i = S.bstart[row + g.lx0]; i < e; ++i) f(i);
    }
}

__device__ __forceinline__ uint2 abs_q(const TileSmem &S, int2 r)
{
    return make_uint2(S.org.x + (uint32_t)r.x, S.org.y + (uint32_t)r.y);
}

// Apex left of v -> w over the region's staged particles (coordinates tile-relative).
__device__ __forceinline__ int apex_smem(const TileSmem &S, int2 pv, int2 pw, const SRegion &g,
                                         float dmax = 0.f)
{
    const int2 dw = make_int2(pw.x - pv.x, pw.y - pv.y);
    const float d2cut = dmax > 0.f ? dmax * dmax : 3.4e38f;
    int best = -1;
    int2 db = make_int2(0, 0);
    Circ cb;
    cb.K = cb.P = cb.Q = cb.Pa = cb.Qa = 0.f;
    for_sregion(S, g, [&](int i) {
        const int2 r = S.rq[i];
        const int2 dc = make_int2(r.x - pv.x, r.y - pv.y);
        const float fx = (float)dc.x, fy = (float)dc.y;
        if (fmaf(fx, fx, fy * fy) > d2cut) return;
        if (cross(dw, dc) <= 0) return;
        if (best >= 0) {
            int t = circ_filter(cb, dc);
            if (t == 0)
                t = incircle_exact(dw, db, dc, abs_q(S, pv), abs_q(S, pw),
                                   abs_q(S, make_int2(db.x + pv.x, db.y + pv.y)), abs_q(S, r));
            if (t < 0) return;
        }
        best = i;
        db = dc;
        cb = make_circ(dw, dc);
    });
    if (best < 0) return -1;
    const float inv2k = 0.5f / cb.K;
    const float cx = -cb.P * inv2k, cy = -cb.Q * inv2k;
    const float r = sqrtf(fmaf(cx, cx, cy * cy));
    const float ext = r + 1e-5f * (cb.Pa + cb.Qa) * (2.f * inv2k) + 64.f;
    if (cx - ext < -g.cl_lo_x || cx + ext > g.cl_hi_x || cy - ext < -g.cl_lo_y ||
        cy + ext > g.cl_hi_y)
        return -1;
    if (dmax > 0.f && 2.f * ext > dmax * 0.9999f) return -1;
    return best;
}

// Star of staged particle v into out[] (staged indices); count, or -PFEM_ERR_* (-1 when the
// star cannot be certified inside the window).
// Star of staged particle v into out[] (staged indices) by gift-wrapping, starting at its
// nearest neighbour; count, or -PFEM_ERR_* (-1 when it cannot be certified in the window).
static __device__ __noinline__ int star_smem(const TileSmem &S, int nb, int v, int R0, int rmax,
                                             float dcut, unsigned short *out)
{
    const int2 pv = S.rq[v];
    for (int attempt = 0, R = R0; R <= rmax; ++attempt, R += attempt > 1 ? 1 : 0) {
        const float dmax = attempt == 0 ? dcut : 0.f;
        SRegion g;
        if (!sregion(S, nb, pv, R, g)) return -1;
        int u0 = -1, gs0 = 0;
        long long d2b = 0x7fffffffffffffffLL;
        bool dup = false;
        for_sregion(S, g, [&](int i) {
            if (i == v) return;
            const int2 r = S.rq[i];
            const long long dx = r.x - pv.x, dy = r.y - pv.y;
            const long long d2 = dx * dx + dy * dy;
            dup |= d2 == 0;
            const int gs = S.gslot[i];
            if (d2 < d2b || (d2 == d2b && gs < gs0)) {
                d2b = d2;
                u0 = i;
                gs0 = gs;
            }
        });
        if (dup) return -PFEM_ERR_DEGENERATE;
        if (u0 < 0) continue;
        int cur = u0, cnt = 0;
        bool ok = true;
        for (;;) {
            if (cnt == KMAX) return -PFEM_ERR_CAPACITY;
            out[cnt++] = (unsigned short)cur;
            const int a = apex_smem(S, pv, S.rq[cur], g, dmax);
            if (a < 0) { ok = false; break; }
            if (a == u0) break;
            cur = a;
        }
        if (ok && cnt >= 3) return cnt;
    }
    return -1;
}

// Claim a star slot for staged particle p (once per tile); false when the table is full.
__device__ __forceinline__ void claim_star(TileSmem &S, int p)
{
    if (atomicCAS((unsigned short *)&S.sslot[p], (unsigned short)0xffff, (unsigned short)0xfffe) ==
        (unsigned short)0xffff) {
        const int w = atomicAdd(&S.nwork, 1);
        if (w < TMAXS) S.work[w] = p;
    }
}

// Star accessor for edge_weights_sa: staged indices mapped to global slots.
struct SmemStar {
    const unsigned short *p;
    const int *gslot;
    int n;
    __device__ __forceinline__ int operator[](int i) const { return gslot[p[i]]; }
};

template <typename P, typename V, typename R, typename SV, bool REFINE, int SHAPE>
__device__ __noinline__ void p2m_node_global(const P2MArgs a, int I, int J)
{
    p2m_node<P, V, R, SV, REFINE, SHAPE, false>(a, I, J);
}

template <typename P, typename V, typename R, typename SV, bool REFINE, int SHAPE>
__global__ void __launch_bounds__(TT, 2) k_p2m_tiled(P2MArgs a, int T, int tiles_x)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem &S = *reinterpret_cast<TileSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int n = a.n, nc = n - 1, nb = a.B.nb;
    const int I0 = (blockIdx.x % tiles_x) * T, J0 = (blockIdx.x / tiles_x) * T;
    const int I1 = min(I0 + T, n) - 1, J1 = min(J0 + T, n) - 1;

    // ---- window
    if (tid == 0) {
        auto ubin = [&](int I) {
            return (long long)bin_of(node_fx(I % nc, nc), nb) + (I >= nc ? nb : 0);
        };
        S.Xo = (long long)node_fx(I0 % nc, nc) + (I0 >= nc ? (1LL << 32) : 0);
        S.Yo = (long long)node_fx(J0 % nc, nc) + (J0 >= nc ? (1LL << 32) : 0);
        S.org = make_uint2(node_fx(I0 % nc, nc), node_fx(J0 % nc, nc));
        S.bx0 = (int)(ubin(I0) - THB);
        S.by0 = (int)(ubin(J0) - THB);
        S.wbx = (int)(ubin(I1) + THB - S.bx0 + 1);
        S.wby = (int)(ubin(J1) + THB - S.by0 + 1);
        S.bad = (S.wbx * S.wby > TMAXB || 2 * S.wbx > nb || 2 * S.wby > nb) ? 1 : 0;
        S.nwork = 0;
    }
    __syncthreads();
    const int nbins = S.bad ? 0 : S.wbx * S.wby;

    // ---- stage the window's particles: 4 consecutive local bins per thread
    int cnt4[4], base = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int b = tid * 4 + k;
        cnt4[k] = 0;
        if (b < nbins) {
            int gx = S.bx0 + b % S.wbx, gy = S.by0 + b / S.wbx;
            gx = ((gx % nb) + nb) % nb;
            gy = ((gy % nb) + nb) % nb;
            const long long gb = (long long)gy * nb + gx;
            cnt4[k] = __ldg(a.B.start + gb + 1) - __ldg(a.B.start + gb);
        }
        tot += cnt4[k];
    }
    {
        const int lane = tid & 31, wid = tid >> 5;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) S.scan[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int w = 0; w < TT / 32; ++w) {
                const int t = S.scan[w];
                S.scan[w] = run;
                run += t;
            }
            S.np = run;
            if (run > TMAXP) S.bad = 1;
        }
        __syncthreads();
        base = S.scan[wid] + incl - tot;
    }
    const bool bad = S.bad != 0;
    if (!bad) {
        int off = base;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = tid * 4 + k;
            if (b < nbins) {
                S.bstart[b] = (unsigned short)off;
                int gx = S.bx0 + b % S.wbx, gy = S.by0 + b / S.wbx;
                gx = ((gx % nb) + nb) % nb;
                gy = ((gy % nb) + nb) % nb;
                const int s0 = __ldg(a.B.start + (long long)gy * nb + gx);
                for (int i = 0; i < cnt4[k]; ++i) {
                    const uint2 q = __ldg(a.B.q + s0 + i);
                    S.rq[off + i] = make_int2((int)(q.x - S.org.x), (int)(q.y - S.org.y));
                    S.gslot[off + i] = s0 + i;
                    S.sslot[off + i] = -1;
                }
                off += cnt4[k];
            }
        }
        if (tid == 0) S.bstart[nbins] = (unsigned short)S.np;
    }
    __syncthreads();

    // ---- per node: nearest staged particle
    const int tcols = I1 - I0 + 1;
    const bool has_node = tid < tcols * (J1 - J0 + 1);
    const int I = I0 + (has_node ? tid % tcols : 0), J = J0 + (has_node ? tid / tcols : 0);
    const int Iu = I % nc, Ju = J % nc;
    bool fallback = bad;
    int v0 = -1;
    int2 pn = make_int2(0, 0);
    if (has_node && !bad) {
        pn = make_int2((int)(node_fx(Iu, nc) - S.org.x), (int)(node_fx(Ju, nc) - S.org.y));
        SRegion g;
        if (sregion(S, nb, pn, 1, g)) {
            long long d2b = 0x7fffffffffffffffLL;
            int gs0 = 0;
            for_sregion(S, g, [&](int i) {
                const int2 r = S.rq[i];
                const long long dx = r.x - pn.x, dy = r.y - pn.y;
                const long long d2 = dx * dx + dy * dy;
                const int gs = S.gslot[i];
                if (d2 < d2b || (d2 == d2b && gs < gs0)) {
                    d2b = d2;
                    v0 = i;
                    gs0 = gs;
                }
            });
            const float clm = fminf(fminf(g.cl_lo_x, g.cl_hi_x), fminf(g.cl_lo_y, g.cl_hi_y));
            if (v0 < 0 || !((float)d2b * 1.0001f < clm * clm)) v0 = -1;
        }
        if (v0 < 0) fallback = true;
        else claim_star(S, v0);
    }
    __syncthreads();

    // ---- stars of the nearest particles
    const int nw1 = min(S.nwork, TMAXS);
    for (int w = tid; w < nw1; w += TT) {
        const int p = S.work[w];
        const int c = star_smem(S, nb, p, a.R0, a.B.rmax, a.B.dmax, S.star[w]);
        S.scount[w] = (signed char)(c < 0 ? (c == -1 ? -1 : c) : c);
        S.sslot[p] = (short)w;
    }
    __syncthreads();

    // ---- locate the node's triangle
    int tri[3] = {-1, -1, -1};
    if (has_node && !fallback) {
        const int sw = S.sslot[v0];
        const int cnt = sw >= 0 ? S.scount[sw] : -1;
        if (cnt < 3) {
            fallback = true;
        } else {
            const unsigned short *st = S.star[sw];
            const int2 q0 = S.rq[v0];
            const int2 dp = make_int2(pn.x - q0.x, pn.y - q0.y);
            if (dp.x == 0 && dp.y == 0) {
                tri[0] = v0; tri[1] = st[0]; tri[2] = st[1];
            } else {
                int j = -1;
                int2 da = make_int2(S.rq[st[cnt - 1]].x - q0.x, S.rq[st[cnt - 1]].y - q0.y);
                for (int k = 0; k < cnt; ++k) {
                    const int2 dn = make_int2(S.rq[st[k]].x - q0.x, S.rq[st[k]].y - q0.y);
                    if (cross(da, dp) >= 0 && cross(dn, dp) < 0) { j = (k + cnt - 1) % cnt; break; }
                    da = dn;
                }
                if (j < 0) {
                    fallback = true;
                } else {
                    int e0 = st[j], e1 = st[(j + 1) % cnt];
                    auto rp = [&](int i) { return make_int2(S.rq[i].x - pn.x, S.rq[i].y - pn.y); };
                    if (cross(rp(e0), rp(e1)) >= 0) {
                        tri[0] = v0; tri[1] = e0; tri[2] = e1;
                    } else {
                        bool done = false;
                        for (int step = 0; step < 64 && !done && !fallback; ++step) {
                            SRegion g;
                            int x = -1;
                            for (int Rr = a.R0; Rr <= a.B.rmax && x < 0; ++Rr) {
                                if (!sregion(S, nb, S.rq[e1], Rr, g)) break;
                                x = apex_smem(S, S.rq[e1], S.rq[e0], g);
                            }
                            if (x < 0) { fallback = true; break; }
                            const int2 pa = rp(e0), pb = rp(e1), pc = rp(x);
                            if (cross(pa, pc) < 0) { e1 = x; continue; }
                            if (cross(pc, pb) < 0) { e0 = x; continue; }
                            tri[0] = e1; tri[1] = e0; tri[2] = x;
                            done = true;
                        }
                        if (!done) fallback = true;
                    }
                }
            }
        }
        if (!fallback && SHAPE == PFEM_SHAPE_QUADRATIC)
            for (int e = 0; e < 3; ++e) claim_star(S, tri[e]);
    }
    __syncthreads();

    // ---- stars of the triangle vertices
    if (SHAPE == PFEM_SHAPE_QUADRATIC) {
        const int nw2 = min(S.nwork, TMAXS);
        for (int w = nw1 + tid; w < nw2; w += TT) {
            const int p = S.work[w];
            const int c = star_smem(S, nb, p, a.R0, a.B.rmax, a.B.dmax, S.star[w]);
            S.scount[w] = (signed char)(c < 0 ? (c == -1 ? -1 : c) : c);
            S.sslot[p] = (short)w;
        }
        __syncthreads();
    }

    if (!has_node) return;
    int sw[3] = {-1, -1, -1};
    if (!fallback && SHAPE == PFEM_SHAPE_QUADRATIC)
        for (int e = 0; e < 3; ++e) {
            sw[e] = S.sslot[tri[e]];
            if (sw[e] < 0 || S.scount[sw[e]] < 3) fallback = true;
        }
    if (fallback) {
        p2m_node_global<P, V, R, SV, REFINE, SHAPE>(a, I, J);
        return;
    }

    // ---- weights and apply
    const long long node = (long long)J * n + I;
    NodePos<P, R> np;
    np.init(Iu, Ju, nc);
    int gt[3];
    R d[3][2];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        gt[e] = S.gslot[tri[e]];
        np.off(a.pos, gt[e], d[e][0], d[e][1]);
    }
    const R area2 = (d[1][0] - d[0][0]) * (d[2][1] - d[0][1]) - (d[1][1] - d[0][1]) * (d[2][0] - d[0][0]);
    const R lam[3] = {(d[1][0] * d[2][1] - d[1][1] * d[2][0]) / area2,
                      (d[2][0] * d[0][1] - d[2][1] * d[0][0]) / area2,
                      (d[0][0] * d[1][1] - d[0][1] * d[1][0]) / area2};
    R acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = R(0);
    auto emit = [&](int s, R wgt) {
        R v[8];
        load_vals<V, R>((const V *)a.vals, a.perm, s, a.C, v);
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < a.C) acc[c] = fma(wgt, v[c], acc[c]);
    };
    int err = 0;
    if (SHAPE == PFEM_SHAPE_QUADRATIC) {
        const SmemStar sa[3] = {{S.star[sw[0]], S.gslot, S.scount[sw[0]]},
                                {S.star[sw[1]], S.gslot, S.scount[sw[1]]},
                                {S.star[sw[2]], S.gslot, S.scount[sw[2]]}};
        err = node_quadratic<P, R, SV, REFINE>(a, np, gt, sa, lam, emit);
    } else {
        for (int e = 0; e < 3; ++e) emit(gt[e], lam[e]);
    }
    err = defer_or_error(a, err, node);
    if (err) {
        if (err < 0) record_error(a.status, -err, node);
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = (R)nan_of<R>();
    }
    store_vals<V, R>((V *)a.out, node, a.C, acc);
}

}  // namespace pfem
