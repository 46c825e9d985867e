/*
 * pfem_oracle.c -- plain, slow FP64 CPU oracle for the 2D particle <-> fixed-mesh
 * projection round trip of Duque & Espanol, "Rapid convergence for simulations that
 * project from particles onto a fixed mesh" (arXiv 1610.05266).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this library.  It shares no code with the CUDA path.
 *
 * What it computes, and where the paper defines it:
 *   - P2M, Sec. 2.2 eq. (p2m): alpha_i = sum_mu alpha_mu psi_mu(r_i) at every mesh node.
 *   - M2P, Sec. 2.2 eq. (m2p): alpha_mu = sum_i alpha_i psi^m_i(r_mu) with linear FE
 *     shape functions on the fixed structured triangular mesh.
 *   - Linear FE shape functions on the particles' Delaunay triangulation, App. B
 *     eqs. (C0), (C1) and the Delaunay definition that follows them.
 *   - Quadratically consistent shape functions, App. B eq. (phiquad):
 *     psi_mu = phi_mu + sum_{nu sigma} A_{mu nu sigma} phi_nu phi_sigma, with A symmetric in
 *     (nu, sigma), zero unless (nu, sigma) is a Delaunay edge, and the A for one edge found
 *     as the minimum-norm solution (App. A: SVD with rank detection) of eqs. (A0), (A1),
 *     (condquad) over the stencil S_e = closed Delaunay 1-rings of nu and sigma.
 *   - Derivatives of P2M with respect to particle positions by the complex-step method
 *     (Squire & Trapp 1998) with the topology held fixed; of M2P by the gradient of the
 *     linear FE field.
 *
 * Readings where the paper is silent (each is a stated choice, mirrored in the design notes):
 *   - Domain is the unit periodic square.  Topology (cells, Delaunay, point location)
 *     uses 32-bit fixed-point coordinates q = round(x * 2^32) mod 2^32; differences of
 *     fixed-point coordinates taken as signed 32-bit give the minimal image.
 *   - Delaunay ties (four cocircular particles) are broken by perturbing the lifted
 *     heights |r|^2 by infinitesimals ordered by the key (qy << 32 | qx): the particle
 *     with the largest key carries the dominant perturbation.
 *   - Arithmetic (barycentrics, moments, weights) uses the caller's FP64 positions as
 *     minimal-image differences from the node.
 *   - The stencil of edge (nu, sigma) is {nu, sigma} + Delaunay neighbours of nu + those
 *     of sigma; A_mu = p_mu . y with p_mu = [1, x, y, x^2, xy, y^2] in coordinates centred
 *     at the edge midpoint and scaled by the edge length (A does not depend on the frame,
 *     eq. (A2_2)); rank threshold sigma_k <= max(k, 6) * eps * sigma_max.
 *   - Each unordered edge of the containing triangle contributes 2 lambda_nu lambda_sigma A
 *     because eq. (phiquad) sums over ordered pairs.
 *   - Mesh triangles split every cell along the (i,j)->(i+1,j+1) diagonal.
 *
 * Method: the Delaunay triangulation around a query point is built by Bowyer-Watson
 * insertion of every particle within a square window (exact integer predicates), and a
 * triangle is trusted only if its circumcircle lies inside the window, so that no particle
 * outside the window can be inside it; otherwise the window grows.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_CAPACITY = 4, OR_ERR_DEGENERATE = 5 };

#define OR_KSTAR 32      /* max Delaunay neighbours kept per particle */
#define OR_KSTEN 96      /* max stencil size of one edge */
#define OR_KNODE 128     /* max distinct particles in one node's weight set */

/* ------------------------------------------------------------------ fixed point */

static uint32_t fx_of(double x) { return (uint32_t)(int64_t)nearbyint(ldexp(x, 32)); }

/* Node I of a periodic mesh with nc = n-1 cells per side: round(I * 2^32 / nc) mod 2^32. */
static uint32_t fx_node(int64_t I, int nc)
{
    return (uint32_t)((((uint64_t)I << 32) + (uint64_t)(nc / 2)) / (uint64_t)nc);
}

static int cell_of(uint32_t q, int nc) { return (int)(((uint64_t)q * (uint64_t)nc) >> 32); }

static double wrap_unit(double d) { return d - nearbyint(d); }

/* ------------------------------------------------------------------ cell list (a1, a2) */

/* Stable counting sort of particles by mesh cell: slots ordered by (cell, original index). */
int or_build_cells(int n, int64_t N, const double *pos, int32_t *cell_start, int32_t *perm,
                   uint32_t *qs)
{
    if (n < 3 || N < 0) return OR_ERR_ARG;
    int nc = n - 1;
    int64_t ncell = (int64_t)nc * nc;
    int32_t *cellid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    int64_t *fill = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = 0;
    for (int64_t m = 0; m < N; ++m) {
        uint32_t qx = fx_of(pos[2 * m]), qy = fx_of(pos[2 * m + 1]);
        int c = cell_of(qy, nc) * nc + cell_of(qx, nc);
        cellid[m] = c;
        fill[c + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) fill[c + 1] += fill[c];
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = (int32_t)fill[c];
    for (int64_t m = 0; m < N; ++m) {
        int64_t slot = fill[cellid[m]]++;
        perm[slot] = (int32_t)m;
        qs[2 * slot] = fx_of(pos[2 * m]);
        qs[2 * slot + 1] = fx_of(pos[2 * m + 1]);
    }
    free(cellid);
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------------------ exact predicates */

typedef struct {
    int64_t x, y;      /* fixed-point coordinates relative to the window centre */
    uint64_t key;      /* (qy << 32) | qx: total order for the tie-break */
    int32_t slot;      /* sorted slot of the particle; -1,-2,-3 for the bounding triangle */
} Pt;

/* Does a carry a larger perturbation than b?  Real particles always beat the three
 * bounding-triangle vertices. */
static int dominates(const Pt *a, const Pt *b)
{
    if (a->slot < 0 || b->slot < 0) {
        if (a->slot < 0 && b->slot < 0) return a->slot > b->slot;
        return b->slot < 0;
    }
    return a->key > b->key;
}

static int sgn128(i128 v) { return (v > 0) - (v < 0); }

/* Sign of det[[1,ax,ay],[1,bx,by],[1,cx,cy]]: > 0 when a, b, c turn counter-clockwise. */
static int orient(const Pt *a, const Pt *b, const Pt *c)
{
    i128 d = (i128)(b->x - a->x) * (c->y - a->y) - (i128)(b->y - a->y) * (c->x - a->x);
    return sgn128(d);
}

/* Exact sign of the incircle determinant, > 0 when d is strictly inside the circle through
 * the counter-clockwise triangle a, b, c.  Differences are below 2^33 in magnitude, so every
 * lifted length l < 2^67 and every cross term |c| < 2^67; l is split as lh*2^34 + ll and
 * the two partial sums are kept in 128-bit integers. */
static int incircle_exact(const Pt *a, const Pt *b, const Pt *c, const Pt *d)
{
    i128 adx = a->x - d->x, ady = a->y - d->y;
    i128 bdx = b->x - d->x, bdy = b->y - d->y;
    i128 cdx = c->x - d->x, cdy = c->y - d->y;
    i128 l[3] = {adx * adx + ady * ady, bdx * bdx + bdy * bdy, cdx * cdx + cdy * cdy};
    i128 k[3] = {bdx * cdy - bdy * cdx, cdx * ady - cdy * adx, adx * bdy - ady * bdx};
    const i128 mask = (((i128)1) << 34) - 1;
    i128 hi = 0, lo = 0;
    for (int t = 0; t < 3; ++t) {
        hi += (l[t] >> 34) * k[t];
        lo += (l[t] & mask) * k[t];
    }
    i128 q = lo >> 34;            /* floor division (arithmetic shift) */
    i128 r = lo - (q << 34);      /* 0 <= r < 2^34 */
    hi += q;
    if (hi != 0) return sgn128(hi);
    return r > 0;
}

/* Incircle with the symbolic tie-break: when d lies exactly on the circle, the point with
 * the largest key is lifted by the dominant infinitesimal.  Lifting point p changes the
 * 4x4 lifted determinant by its cofactor, which is an orientation of the other three. */
static int incircle(const Pt *a, const Pt *b, const Pt *c, const Pt *d)
{
    int s = incircle_exact(a, b, c, d);
    if (s) return s;
    const Pt *pts[4] = {a, b, c, d};
    int m = 0;
    for (int t = 1; t < 4; ++t)
        if (dominates(pts[t], pts[m])) m = t;
    switch (m) {
    case 0: return orient(b, c, d);
    case 1: return -orient(a, c, d);
    case 2: return orient(a, b, d);
    default: return -orient(a, b, c);
    }
}

/* ------------------------------------------------------------------ window triangulation */

typedef struct { int v[3]; int alive; } Tri;

typedef struct {
    Pt *p; int np, capp;
    Tri *t; int nt, capt;
    int *bad; int capbad;
    int64_t W;               /* window half-width in fixed-point units */
} Win;

static void win_free(Win *w)
{
    free(w->p); free(w->t); free(w->bad);
    memset(w, 0, sizeof(*w));
}

static void win_reserve(Win *w, int np)
{
    if (np + 3 > w->capp) {
        w->capp = 2 * (np + 3);
        w->p = (Pt *)realloc(w->p, sizeof(Pt) * (size_t)w->capp);
    }
    int nt = 2 * (np + 3) + 16;
    if (nt * 4 > w->capt) {
        w->capt = nt * 4;
        w->t = (Tri *)realloc(w->t, sizeof(Tri) * (size_t)w->capt);
    }
    if (nt > w->capbad) {
        w->capbad = nt * 4;
        w->bad = (int *)realloc(w->bad, sizeof(int) * (size_t)w->capbad);
    }
}

static void add_tri(Win *w, int a, int b, int c)
{
    if (w->nt == w->capt) {
        w->capt *= 2;
        w->t = (Tri *)realloc(w->t, sizeof(Tri) * (size_t)w->capt);
    }
    Tri *t = &w->t[w->nt++];
    t->v[0] = a; t->v[1] = b; t->v[2] = c; t->alive = 1;
}

/* Bowyer-Watson insertion of point pi: delete every triangle whose (perturbed) circumcircle
 * contains it and fan the hole's boundary to the new point. */
static int bw_insert(Win *w, int pi)
{
    int nb = 0;
    for (int t = 0; t < w->nt; ++t) {
        Tri *T = &w->t[t];
        if (!T->alive) continue;
        if (incircle(&w->p[T->v[0]], &w->p[T->v[1]], &w->p[T->v[2]], &w->p[pi]) > 0) {
            if (nb == w->capbad) {
                w->capbad *= 2;
                w->bad = (int *)realloc(w->bad, sizeof(int) * (size_t)w->capbad);
            }
            w->bad[nb++] = t;
        }
    }
    if (nb == 0) return OR_ERR_DEGENERATE;
    int nt0 = w->nt;
    for (int i = 0; i < nb; ++i) {
        Tri *T = &w->t[w->bad[i]];
        for (int e = 0; e < 3; ++e) {
            int u = T->v[e], v = T->v[(e + 1) % 3];
            int shared = 0;
            for (int j = 0; j < nb && !shared; ++j) {
                if (j == i) continue;
                Tri *S = &w->t[w->bad[j]];
                for (int f = 0; f < 3; ++f)
                    if (S->v[f] == v && S->v[(f + 1) % 3] == u) { shared = 1; break; }
            }
            if (!shared) add_tri(w, u, v, pi);
        }
    }
    for (int i = 0; i < nb; ++i) w->t[w->bad[i]].alive = 0;
    /* compact: drop dead triangles so later scans stay short */
    int k = 0;
    for (int t = 0; t < w->nt; ++t)
        if (w->t[t].alive) w->t[k++] = w->t[t];
    (void)nt0;
    w->nt = k;
    return OR_OK;
}

typedef struct {
    int n, nc;
    int64_t N;
    const double *pos;          /* [N,2] caller positions (FP64) */
    const int32_t *cell_start;
    const int32_t *perm;
    const uint32_t *qs;         /* [N,2] sorted fixed-point coordinates */
} Geo;

/* Collect every particle with |dx|,|dy| <= W around fixed-point centre (cx, cy) and
 * triangulate them inside a bounding triangle.  Returns OR_ERR_DEGENERATE on duplicates. */
static int win_build(Win *w, const Geo *g, uint32_t cx, uint32_t cy, int64_t W)
{
    int nc = g->nc;
    int64_t cellw = ((int64_t)1 << 32) / nc + 1;    /* cell width in fixed-point units */
    int r = (int)(W / cellw) + 1;
    int ccx = cell_of(cx, nc), ccy = cell_of(cy, nc);
    int spanx = 2 * r + 1 >= nc ? nc : 2 * r + 1;
    int spany = spanx;
    int x0 = 2 * r + 1 >= nc ? 0 : ccx - r;
    int y0 = 2 * r + 1 >= nc ? 0 : ccy - r;
    w->np = 0;
    w->nt = 0;
    w->W = W;
    for (int pass = 0; pass < 2; ++pass) {
        int cnt = 0;
        for (int oy = 0; oy < spany; ++oy) {
            int cy_ = ((y0 + oy) % nc + nc) % nc;
            for (int ox = 0; ox < spanx; ++ox) {
                int cx_ = ((x0 + ox) % nc + nc) % nc;
                int c = cy_ * nc + cx_;
                for (int32_t s = g->cell_start[c]; s < g->cell_start[c + 1]; ++s) {
                    int64_t dx = (int32_t)(g->qs[2 * s] - cx);
                    int64_t dy = (int32_t)(g->qs[2 * s + 1] - cy);
                    if (dx > W || dx < -W || dy > W || dy < -W) continue;
                    if (pass == 1) {
                        Pt *P = &w->p[3 + cnt];
                        P->x = dx; P->y = dy;
                        P->key = ((uint64_t)g->qs[2 * s + 1] << 32) | g->qs[2 * s];
                        P->slot = s;
                    }
                    ++cnt;
                }
            }
        }
        if (pass == 0) win_reserve(w, cnt);
        else w->np = cnt + 3;
    }
    /* bounding triangle well outside the window square */
    Pt *S = w->p;
    S[0].x = -4 * W; S[0].y = -2 * W; S[0].key = 0; S[0].slot = -3;
    S[1].x = 4 * W;  S[1].y = -2 * W; S[1].key = 0; S[1].slot = -2;
    S[2].x = 0;      S[2].y = 4 * W;  S[2].key = 0; S[2].slot = -1;
    add_tri(w, 0, 1, 2);
    for (int i = 3; i < w->np; ++i) {
        for (int j = 3; j < i; ++j)
            if (w->p[j].x == w->p[i].x && w->p[j].y == w->p[i].y) return OR_ERR_DEGENERATE;
        int st = bw_insert(w, i);
        if (st) return st;
    }
    return OR_OK;
}

/* A triangle is trusted when it has no bounding vertex and its circumcircle lies inside
 * the window square with a margin, so no particle outside the window can be inside it. */
static int tri_trusted(const Win *w, const Tri *T)
{
    const Pt *a = &w->p[T->v[0]], *b = &w->p[T->v[1]], *c = &w->p[T->v[2]];
    if (a->slot < 0 || b->slot < 0 || c->slot < 0) return 0;
    double bx = (double)(b->x - a->x), by = (double)(b->y - a->y);
    double cx = (double)(c->x - a->x), cy = (double)(c->y - a->y);
    double D = 2.0 * (bx * cy - by * cx);
    if (D == 0.0) return 0;
    double b2 = bx * bx + by * by, c2 = cx * cx + cy * cy;
    double ux = (cy * b2 - by * c2) / D, uy = (bx * c2 - cx * b2) / D;
    double R = sqrt(ux * ux + uy * uy);
    double ox = (double)a->x + ux, oy = (double)a->y + uy;
    double lim = (double)w->W * (1.0 - 1e-6) - 16.0;
    return fabs(ox) + R * (1.0 + 1e-9) < lim && fabs(oy) + R * (1.0 + 1e-9) < lim;
}

/* Counter-clockwise Delaunay neighbours of window point v (all incident triangles must be
 * trusted).  Returns the count, or -1. */
static int win_star(const Win *w, int v, int *out, int kmax)
{
    int xs[4 * OR_KSTAR], ys[4 * OR_KSTAR], ninc = 0;
    for (int t = 0; t < w->nt; ++t) {
        const Tri *T = &w->t[t];
        for (int e = 0; e < 3; ++e)
            if (T->v[e] == v) {
                if (ninc == 4 * OR_KSTAR || !tri_trusted(w, T)) return -1;
                /* in the CCW triangle (v, x, y) the fan around v runs from x to y */
                xs[ninc] = T->v[(e + 1) % 3];
                ys[ninc] = T->v[(e + 2) % 3];
                ++ninc;
            }
    }
    if (ninc < 3 || ninc > kmax) return -1;
    int cnt = 0, cur = xs[0];
    do {
        if (cnt >= ninc) return -1;
        out[cnt++] = cur;
        int nxt = -1;
        for (int i = 0; i < ninc; ++i)
            if (xs[i] == cur) { nxt = ys[i]; break; }
        if (nxt < 0) return -1;
        cur = nxt;
    } while (cur != xs[0]);
    return cnt == ninc ? cnt : -1;
}

/* The trusted triangle containing the window centre (origin), or -1. */
static int win_locate(const Win *w)
{
    Pt o; o.x = 0; o.y = 0; o.key = 0; o.slot = 0;
    for (int t = 0; t < w->nt; ++t) {
        const Tri *T = &w->t[t];
        const Pt *a = &w->p[T->v[0]], *b = &w->p[T->v[1]], *c = &w->p[T->v[2]];
        if (orient(a, b, &o) >= 0 && orient(b, c, &o) >= 0 && orient(c, a, &o) >= 0)
            return tri_trusted(w, T) ? t : -1;
    }
    return -1;
}

/* ------------------------------------------------------------------ min-norm solve */

/* Minimum-norm solution of P A = b, P = 6 x k given by its columns pk[j][0..5], through a
 * one-sided (Hestenes) Jacobi SVD of P^T with singular values <= max(k,6) eps sigma_max
 * dropped.  Writes A[0..k).  Returns the numerical rank. */
static int minnorm_svd(int k, double pk[][6], const double b[6], double *A)
{
    double G[OR_KSTEN][6], V[6][6];
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < 6; ++c) G[r][c] = pk[r][c];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) V[i][j] = (i == j);
    for (int sweep = 0; sweep < 80; ++sweep) {
        int rotated = 0;
        for (int i = 0; i < 5; ++i)
            for (int j = i + 1; j < 6; ++j) {
                double al = 0, be = 0, ga = 0;
                for (int r = 0; r < k; ++r) {
                    al += G[r][i] * G[r][i];
                    be += G[r][j] * G[r][j];
                    ga += G[r][i] * G[r][j];
                }
                if (ga == 0.0 || fabs(ga) <= DBL_EPSILON * sqrt(al * be)) continue;
                rotated = 1;
                double zeta = (be - al) / (2.0 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int r = 0; r < k; ++r) {
                    double gi = G[r][i], gj = G[r][j];
                    G[r][i] = cs * gi - sn * gj;
                    G[r][j] = sn * gi + cs * gj;
                }
                for (int r = 0; r < 6; ++r) {
                    double vi = V[r][i], vj = V[r][j];
                    V[r][i] = cs * vi - sn * vj;
                    V[r][j] = sn * vi + cs * vj;
                }
            }
        if (!rotated) break;
    }
    double sig[6], smax = 0;
    for (int c = 0; c < 6; ++c) {
        double s = 0;
        for (int r = 0; r < k; ++r) s += G[r][c] * G[r][c];
        sig[c] = sqrt(s);
        if (sig[c] > smax) smax = sig[c];
    }
    double tol = (k > 6 ? k : 6) * DBL_EPSILON * smax;
    for (int r = 0; r < k; ++r) A[r] = 0;
    int rank = 0;
    /* P^T = U S V^T with U = G S^-1, so A = U S^+ V^T b = sum_c G[:,c] (V[:,c].b) / sig_c^2 */
    for (int c = 0; c < 6; ++c) {
        if (sig[c] <= tol) continue;
        ++rank;
        double vb = 0;
        for (int r = 0; r < 6; ++r) vb += V[r][c] * b[r];
        double f = vb / (sig[c] * sig[c]);
        for (int r = 0; r < k; ++r) A[r] += G[r][c] * f;
    }
    return rank;
}

/* ------------------------------------------------------------------ node weights */

typedef struct {
    int tri[3];          /* window indices of the containing triangle, CCW */
    int star[3][OR_KSTAR];
    int nstar[3];
    Win w;
} NodeQ;

static void particle_offset(const Geo *g, int32_t slot, double xq, double yq, double *dx,
                            double *dy)
{
    int32_t m = g->perm[slot];
    *dx = wrap_unit(g->pos[2 * m] - xq);
    *dy = wrap_unit(g->pos[2 * m + 1] - yq);
}

/* Locate the node (fixed-point qx, qy) in the particle Delaunay triangulation and, when
 * need_stars, collect the stars of the three vertices; the window grows until everything
 * used is trusted. */
static int node_query(const Geo *g, uint32_t qx, uint32_t qy, int need_stars, NodeQ *Q)
{
    double hbar = 4294967296.0 / sqrt((double)(g->N > 0 ? g->N : 1));
    int64_t W = (int64_t)(3.5 * hbar);
    const int64_t Wmax = (int64_t)1 << 30;
    for (;;) {
        if (W > Wmax) W = Wmax;
        int st = win_build(&Q->w, g, qx, qy, W);
        if (st) return st;
        int t = win_locate(&Q->w);
        int ok = t >= 0;
        if (ok) {
            for (int e = 0; e < 3; ++e) Q->tri[e] = Q->w.t[t].v[e];
            if (need_stars)
                for (int e = 0; e < 3 && ok; ++e) {
                    Q->nstar[e] = win_star(&Q->w, Q->tri[e], Q->star[e], OR_KSTAR);
                    ok = Q->nstar[e] >= 3;
                }
        }
        if (ok) return OR_OK;
        if (W == Wmax) return OR_ERR_CAPACITY;
        W = W + W / 2;
    }
}

/* Barycentric coordinates of the origin in triangle with offsets d[3][2]. */
static void barycentric(double d[3][2], double lam[3])
{
    double area2 = (d[1][0] - d[0][0]) * (d[2][1] - d[0][1]) - (d[1][1] - d[0][1]) * (d[2][0] - d[0][0]);
    lam[0] = (d[1][0] * d[2][1] - d[1][1] * d[2][0]) / area2;
    lam[1] = (d[2][0] * d[0][1] - d[2][1] * d[0][0]) / area2;
    lam[2] = (d[0][0] * d[1][1] - d[0][1] * d[1][0]) / area2;
}

/* Stencil of the edge between triangle vertices e and (e+1)%3: both endpoints plus both
 * stars, each particle once.  Returns window indices. */
static int edge_stencil(const NodeQ *Q, int e, int *S)
{
    int f = (e + 1) % 3, k = 0;
    int cand[2 + 2 * OR_KSTAR];
    cand[k++] = Q->tri[e];
    cand[k++] = Q->tri[f];
    for (int i = 0; i < Q->nstar[e]; ++i) cand[k++] = Q->star[e][i];
    for (int i = 0; i < Q->nstar[f]; ++i) cand[k++] = Q->star[f][i];
    int n = 0;
    for (int i = 0; i < k; ++i) {
        int dup = 0;
        for (int j = 0; j < n; ++j)
            if (S[j] == cand[i]) { dup = 1; break; }
        if (!dup) S[n++] = cand[i];
    }
    return n;
}

typedef struct {
    int32_t slot[OR_KNODE];
    double w[OR_KNODE];
    int n;
} WSet;

static void wset_add(WSet *s, int32_t slot, double w)
{
    for (int i = 0; i < s->n; ++i)
        if (s->slot[i] == slot) { s->w[i] += w; return; }
    if (s->n < OR_KNODE) {
        s->slot[s->n] = slot;
        s->w[s->n++] = w;
    }
}

/* A coefficients of one edge (eqs. A0, A1, condquad) over stencil S of size k, with
 * offsets from the node; returns rank. */
static int edge_coeffs(const Geo *g, const Win *w, const int *S, int k, int inu, int isg,
                       double xq, double yq, double *A)
{
    double dnu[2], dsg[2];
    particle_offset(g, w->p[inu].slot, xq, yq, &dnu[0], &dnu[1]);
    particle_offset(g, w->p[isg].slot, xq, yq, &dsg[0], &dsg[1]);
    double mx = 0.5 * (dnu[0] + dsg[0]), my = 0.5 * (dnu[1] + dsg[1]);
    double ex = dnu[0] - dsg[0], ey = dnu[1] - dsg[1];
    double s = sqrt(ex * ex + ey * ey);
    double pk[OR_KSTEN][6];
    for (int i = 0; i < k; ++i) {
        double dx, dy;
        particle_offset(g, w->p[S[i]].slot, xq, yq, &dx, &dy);
        double x = (dx - mx) / s, y = (dy - my) / s;
        pk[i][0] = 1; pk[i][1] = x; pk[i][2] = y;
        pk[i][3] = x * x; pk[i][4] = x * y; pk[i][5] = y * y;
    }
    double tx = ex / s, ty = ey / s;
    double b[6] = {0, 0, 0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
    return minnorm_svd(k, pk, b, A);
}

/* Weights of one mesh node: linear (shape 0) or quadratic (shape 1). */
static int node_weights(const Geo *g, int I, int J, int shape, WSet *out, NodeQ *Q,
                        int *min_rank)
{
    int nc = g->nc;
    int Iu = I % nc, Ju = J % nc;
    double xq = (double)Iu / (double)nc, yq = (double)Ju / (double)nc;
    int st = node_query(g, fx_node(Iu, nc), fx_node(Ju, nc), shape == 1, Q);
    if (st) return st;
    double d[3][2], lam[3];
    for (int e = 0; e < 3; ++e) particle_offset(g, Q->w.p[Q->tri[e]].slot, xq, yq, &d[e][0], &d[e][1]);
    barycentric(d, lam);
    out->n = 0;
    for (int e = 0; e < 3; ++e) wset_add(out, Q->w.p[Q->tri[e]].slot, lam[e]);
    if (min_rank) *min_rank = 6;
    if (shape == 1) {
        for (int e = 0; e < 3; ++e) {
            int f = (e + 1) % 3;
            int S[2 + 2 * OR_KSTAR];
            int k = edge_stencil(Q, e, S);
            double A[OR_KSTEN];
            int rank = edge_coeffs(g, &Q->w, S, k, Q->tri[e], Q->tri[f], xq, yq, A);
            if (min_rank && rank < *min_rank) *min_rank = rank;
            double c = 2.0 * lam[e] * lam[f];
            for (int i = 0; i < k; ++i) wset_add(out, Q->w.p[S[i]].slot, c * A[i]);
        }
    }
    return OR_OK;
}

static Geo make_geo(int n, int64_t N, const double *pos, const int32_t *cs, const int32_t *perm,
                    const uint32_t *qs)
{
    Geo g;
    g.n = n; g.nc = n - 1; g.N = N; g.pos = pos; g.cell_start = cs; g.perm = perm; g.qs = qs;
    return g;
}

/* Weights of node (I, J) as (original particle index, weight) pairs.  Also reports the
 * containing triangle (original indices, CCW) and its barycentrics. */
int or_node_weights(int n, int64_t N, const double *pos, const int32_t *cell_start,
                    const int32_t *perm, const uint32_t *qs, int I, int J, int shape, int kmax,
                    int32_t *idx, double *w, int *count, int32_t *tri, int *min_rank)
{
    Geo g = make_geo(n, N, pos, cell_start, perm, qs);
    NodeQ Q;
    memset(&Q, 0, sizeof(Q));
    WSet s;
    int st = node_weights(&g, I, J, shape, &s, &Q, min_rank);
    if (st == OR_OK) {
        if (s.n > kmax) st = OR_ERR_CAPACITY;
        else {
            for (int i = 0; i < s.n; ++i) { idx[i] = perm[s.slot[i]]; w[i] = s.w[i]; }
            *count = s.n;
            for (int e = 0; e < 3; ++e) tri[e] = perm[Q.w.p[Q.tri[e]].slot];
        }
    }
    win_free(&Q.w);
    return st;
}

/* Per-edge detail for node (I, J): stencil (original indices) and A for each of the three
 * edges (e, e+1) of the containing triangle; lam = barycentrics. */
int or_node_edges(int n, int64_t N, const double *pos, const int32_t *cell_start,
                  const int32_t *perm, const uint32_t *qs, int I, int J, int32_t *tri,
                  double *lam, int32_t *stencil /*[3][OR_KSTEN]*/, double *A /*[3][OR_KSTEN]*/,
                  int *k /*[3]*/, int *rank /*[3]*/)
{
    Geo g = make_geo(n, N, pos, cell_start, perm, qs);
    NodeQ Q;
    memset(&Q, 0, sizeof(Q));
    int nc = n - 1;
    int Iu = I % nc, Ju = J % nc;
    double xq = (double)Iu / nc, yq = (double)Ju / nc;
    int st = node_query(&g, fx_node(Iu, nc), fx_node(Ju, nc), 1, &Q);
    if (st == OR_OK) {
        double d[3][2];
        for (int e = 0; e < 3; ++e) particle_offset(&g, Q.w.p[Q.tri[e]].slot, xq, yq, &d[e][0], &d[e][1]);
        barycentric(d, lam);
        for (int e = 0; e < 3; ++e) {
            tri[e] = perm[Q.w.p[Q.tri[e]].slot];
            int S[2 + 2 * OR_KSTAR];
            int kk = edge_stencil(&Q, e, S);
            rank[e] = edge_coeffs(&g, &Q.w, S, kk, Q.tri[e], Q.tri[(e + 1) % 3], xq, yq, A + e * OR_KSTEN);
            k[e] = kk;
            for (int i = 0; i < kk; ++i) stencil[e * OR_KSTEN + i] = perm[Q.w.p[S[i]].slot];
        }
    }
    win_free(&Q.w);
    return st;
}

/* Counter-clockwise Delaunay neighbours (original indices) of original particle m. */
int or_star(int n, int64_t N, const double *pos, const int32_t *cell_start, const int32_t *perm,
            const uint32_t *qs, int64_t m, int32_t *out, int kmax, int *count)
{
    Geo g = make_geo(n, N, pos, cell_start, perm, qs);
    int32_t slot = -1;
    for (int64_t s = 0; s < N; ++s)
        if (perm[s] == m) { slot = (int32_t)s; break; }
    if (slot < 0) return OR_ERR_ARG;
    uint32_t cx = qs[2 * slot], cy = qs[2 * slot + 1];
    Win w;
    memset(&w, 0, sizeof(w));
    double hbar = 4294967296.0 / sqrt((double)N);
    int64_t W = (int64_t)(3.0 * hbar);
    const int64_t Wmax = (int64_t)1 << 30;
    int st = OR_ERR_CAPACITY;
    for (;;) {
        if (W > Wmax) W = Wmax;
        int b = win_build(&w, &g, cx, cy, W);
        if (b) { st = b; break; }
        int v = -1;
        for (int i = 3; i < w.np; ++i)
            if (w.p[i].slot == slot) { v = i; break; }
        int buf[OR_KSTAR];
        int c = v >= 0 ? win_star(&w, v, buf, OR_KSTAR) : -1;
        if (c >= 3) {
            if (c > kmax) { st = OR_ERR_CAPACITY; break; }
            for (int i = 0; i < c; ++i) out[i] = perm[w.p[buf[i]].slot];
            *count = c;
            st = OR_OK;
            break;
        }
        if (W == Wmax) break;
        W = W + W / 2;
    }
    win_free(&w);
    return st;
}

/* ------------------------------------------------------------------ P2M and M2P */

static void *xcalloc(size_t n, size_t s) { return calloc(n ? n : 1, s); }

/* P2M (eq. p2m) for all n x n nodes, image row and column included. */
int or_p2m(int n, int64_t N, const double *pos, int C, const double *vals, int shape,
           double *mesh, int nthreads, int64_t node_begin, int64_t node_end)
{
    if (n < 3 || N < 3 || C < 1) return OR_ERR_ARG;
    int64_t ncell = (int64_t)(n - 1) * (n - 1);
    int32_t *cs = (int32_t *)xcalloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t *perm = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    uint32_t *qs = (uint32_t *)xcalloc((size_t)N * 2, sizeof(uint32_t));
    or_build_cells(n, N, pos, cs, perm, qs);
    Geo g = make_geo(n, N, pos, cs, perm, qs);
    int64_t nn = (int64_t)n * n;
    if (node_end < 0 || node_end > nn) node_end = nn;
    if (node_begin < 0 || node_begin > node_end) {
        free(cs); free(perm); free(qs);
        return OR_ERR_ARG;
    }
    int err = OR_OK;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        NodeQ Q;
        memset(&Q, 0, sizeof(Q));
        WSet s;
#pragma omp for schedule(dynamic, 16)
        for (int64_t node = node_begin; node < node_end; ++node) {
            int J = (int)(node / n), I = (int)(node % n);
            int st = node_weights(&g, I, J, shape, &s, &Q, NULL);
            if (st) {
#pragma omp atomic write
                err = st;
                continue;
            }
            for (int c = 0; c < C; ++c) {
                double acc = 0;
                for (int i = 0; i < s.n; ++i) acc += s.w[i] * vals[(int64_t)perm[s.slot[i]] * C + c];
                mesh[node * C + c] = acc;
            }
        }
        win_free(&Q.w);
    }
    free(cs); free(perm); free(qs);
    return err;
}

/* Mesh-triangle weights of a point: cell (i,j) from the fixed-point coordinates, local
 * (s,t) from the FP64 offset to the cell corner. */
static void m2p_weights(int n, double x, double y, int64_t node[3], double wgt[3], int *ci,
                        int *cj, double *s_out, double *t_out)
{
    int nc = n - 1;
    int i = cell_of(fx_of(x), nc), j = cell_of(fx_of(y), nc);
    double s = wrap_unit(x - (double)i / nc) * nc;
    double t = wrap_unit(y - (double)j / nc) * nc;
    if (s >= t) {
        node[0] = (int64_t)j * n + i; wgt[0] = 1 - s;
        node[1] = (int64_t)j * n + i + 1; wgt[1] = s - t;
        node[2] = (int64_t)(j + 1) * n + i + 1; wgt[2] = t;
    } else {
        node[0] = (int64_t)j * n + i; wgt[0] = 1 - t;
        node[1] = (int64_t)(j + 1) * n + i + 1; wgt[1] = s;
        node[2] = (int64_t)(j + 1) * n + i; wgt[2] = t - s;
    }
    *ci = i; *cj = j; *s_out = s; *t_out = t;
}

/* M2P (eq. m2p) with linear FE on the structured mesh. */
int or_m2p(int n, int64_t N, const double *pos, int C, const double *mesh, double *vals)
{
    if (n < 3 || N < 0 || C < 1) return OR_ERR_ARG;
    for (int64_t m = 0; m < N; ++m) {
        int64_t node[3]; double w[3]; int i, j; double s, t;
        m2p_weights(n, pos[2 * m], pos[2 * m + 1], node, w, &i, &j, &s, &t);
        for (int c = 0; c < C; ++c)
            vals[m * C + c] = w[0] * mesh[node[0] * C + c] + w[1] * mesh[node[1] * C + c] +
                              w[2] * mesh[node[2] * C + c];
    }
    return OR_OK;
}

/* Adjoint of M2P: grad_mesh[node] = sum over particles of W * g (into the stored entry the
 * forward read), grad_pos = g . grad of the linear FE field at the particle. */
int or_m2p_backward(int n, int64_t N, const double *pos, int C, const double *mesh,
                    const double *grad_vals, double *grad_mesh, double *grad_pos)
{
    int64_t nn = (int64_t)n * n;
    for (int64_t i = 0; i < nn * C; ++i) grad_mesh[i] = 0;
    int nc = n - 1;
    for (int64_t m = 0; m < N; ++m) {
        int64_t node[3]; double w[3]; int i, j; double s, t;
        m2p_weights(n, pos[2 * m], pos[2 * m + 1], node, w, &i, &j, &s, &t);
        double gx = 0, gy = 0;
        int64_t n00 = (int64_t)j * n + i, n10 = n00 + 1, n11 = n00 + n + 1, n01 = n00 + n;
        for (int c = 0; c < C; ++c) {
            double g = grad_vals[m * C + c];
            for (int e = 0; e < 3; ++e) grad_mesh[node[e] * C + c] += w[e] * g;
            double f00 = mesh[n00 * C + c], f10 = mesh[n10 * C + c];
            double f11 = mesh[n11 * C + c], f01 = mesh[n01 * C + c];
            double ds, dt;
            if (s >= t) { ds = f10 - f00; dt = f11 - f10; }
            else { ds = f11 - f01; dt = f01 - f00; }
            gx += g * ds * nc;
            gy += g * dt * nc;
        }
        grad_pos[2 * m] = gx;
        grad_pos[2 * m + 1] = gy;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ mesh QCSF (M2P)
 *
 * Quadratically consistent shape functions on the fixed mesh (App. B applied to the mesh
 * triangulation; the paper's projFEM6 and projFEMq interpolate mesh -> particles with them,
 * Table 1, and compute their geometric coefficients once, Sec. 3.1).  Every cell is split
 * along (i,j)->(i+1,j+1), so node (I,J) has the six neighbours (I+-1,J), (I,J+-1), (I+1,J+1),
 * (I-1,J-1).  An edge's stencil is the closed neighbourhood of both endpoints (10 nodes) and
 * its coefficients are the minimum-norm solution of eqs. A0, A1, condquad; on the uniform
 * mesh they depend only on the edge's direction: (1,0), (0,1) or (1,1). */

static const int MESH_NB[6][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, -1}};

/* Stencil (node offsets from the edge's first node) and coefficients of the mesh edge from
 * (0,0) to (ex,ey). */
static int mesh_edge(int ex, int ey, int S[16][2], double A[16])
{
    int k = 0;
    int ends[2][2] = {{0, 0}, {ex, ey}};
    for (int e = 0; e < 2; ++e)
        for (int m = -1; m < 6; ++m) {
            int x = ends[e][0] + (m < 0 ? 0 : MESH_NB[m][0]);
            int y = ends[e][1] + (m < 0 ? 0 : MESH_NB[m][1]);
            int dup = 0;
            for (int i = 0; i < k; ++i)
                if (S[i][0] == x && S[i][1] == y) dup = 1;
            if (!dup) { S[k][0] = x; S[k][1] = y; ++k; }
        }
    double s = sqrt((double)(ex * ex + ey * ey));
    double pk[OR_KSTEN][6];
    for (int i = 0; i < k; ++i) {
        double x = (S[i][0] - 0.5 * ex) / s, y = (S[i][1] - 0.5 * ey) / s;
        pk[i][0] = 1; pk[i][1] = x; pk[i][2] = y; pk[i][3] = x * x; pk[i][4] = x * y; pk[i][5] = y * y;
    }
    double tx = ex / s, ty = ey / s;
    double b[6] = {0, 0, 0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
    minnorm_svd(k, pk, b, A);
    return k;
}

/* Stencil and coefficients of a mesh edge type: 0 = (1,0), 1 = (0,1), 2 = (1,1). */
int or_mesh_edge(int type, int32_t *offsets /*[16][2]*/, double *A /*[16]*/)
{
    static const int D[3][2] = {{1, 0}, {0, 1}, {1, 1}};
    if (type < 0 || type > 2) return -1;
    int S[16][2];
    int k = mesh_edge(D[type][0], D[type][1], S, A);
    for (int i = 0; i < k; ++i) { offsets[2 * i] = S[i][0]; offsets[2 * i + 1] = S[i][1]; }
    return k;
}

/* M2P with mesh QCSF: alpha_mu = sum_i w_i alpha_i, w_i = lambda_i [i in T] +
 * sum over the edges (P, Q) of T of 2 lambda_P lambda_Q A_{i,(P,Q)} (eq. phiquad on the mesh).
 * Node values are read at unique nodes (I mod (n-1), J mod (n-1)). */
int or_m2p_quadratic(int n, int64_t N, const double *pos, int C, const double *mesh, double *vals)
{
    if (n < 3 || N < 0 || C < 1) return OR_ERR_ARG;
    int nc = n - 1;
    int S[3][16][2];
    double A[3][16];
    int K[3];
    static const int D[3][2] = {{1, 0}, {0, 1}, {1, 1}};
    for (int t = 0; t < 3; ++t) K[t] = mesh_edge(D[t][0], D[t][1], S[t], A[t]);
    for (int64_t m = 0; m < N; ++m) {
        double x = pos[2 * m], y = pos[2 * m + 1];
        int i = cell_of(fx_of(x), nc), j = cell_of(fx_of(y), nc);
        double s = wrap_unit(x - (double)i / nc) * nc;
        double t = wrap_unit(y - (double)j / nc) * nc;
        int V[3][2];
        double lam[3];
        if (s >= t) {
            V[0][0] = 0; V[0][1] = 0; V[1][0] = 1; V[1][1] = 0; V[2][0] = 1; V[2][1] = 1;
            lam[0] = 1 - s; lam[1] = s - t; lam[2] = t;
        } else {
            V[0][0] = 0; V[0][1] = 0; V[1][0] = 1; V[1][1] = 1; V[2][0] = 0; V[2][1] = 1;
            lam[0] = 1 - t; lam[1] = s; lam[2] = t - s;
        }
        for (int c = 0; c < C; ++c) vals[m * C + c] = 0;
        for (int e = 0; e < 3; ++e) {
            int I = ((i + V[e][0]) % nc + nc) % nc, J = ((j + V[e][1]) % nc + nc) % nc;
            for (int c = 0; c < C; ++c) vals[m * C + c] += lam[e] * mesh[((int64_t)J * n + I) * C + c];
        }
        for (int e = 0; e < 3; ++e) {
            int f = (e + 1) % 3;
            int dx = V[f][0] - V[e][0], dy = V[f][1] - V[e][1];
            int bx = V[e][0], by = V[e][1];
            if (dx < 0 || dy < 0) { dx = -dx; dy = -dy; bx = V[f][0]; by = V[f][1]; }
            int type = (dx == 1 && dy == 0) ? 0 : (dx == 0 && dy == 1) ? 1 : 2;
            double cf = 2.0 * lam[e] * lam[f];
            for (int k = 0; k < K[type]; ++k) {
                int I = ((i + bx + S[type][k][0]) % nc + nc) % nc;
                int J = ((j + by + S[type][k][1]) % nc + nc) % nc;
                for (int c = 0; c < C; ++c)
                    vals[m * C + c] += cf * A[type][k] * mesh[((int64_t)J * n + I) * C + c];
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ complex step */

typedef double _Complex cplx;

static cplx cmk(double re, double im) { return __builtin_complex(re, im); }

typedef struct {
    int32_t slot[OR_KNODE];
    cplx w[OR_KNODE];
    int n;
} CSet;

static void cset_add(CSet *s, int32_t slot, cplx w)
{
    for (int i = 0; i < s->n; ++i)
        if (s->slot[i] == slot) { s->w[i] += w; return; }
    if (s->n < OR_KNODE) {
        s->slot[s->n] = slot;
        s->w[s->n++] = w;
    }
}

/* Offset of a window particle from the node with an imaginary part h on coordinate `dim`
 * of the particle with sorted slot `kslot`. */
static void coffset(const Geo *g, int32_t slot, double xq, double yq, int32_t kslot, int dim,
                    double h, cplx *dx, cplx *dy)
{
    double rx, ry;
    particle_offset(g, slot, xq, yq, &rx, &ry);
    *dx = cmk(rx, (slot == kslot && dim == 0) ? h : 0.0);
    *dy = cmk(ry, (slot == kslot && dim == 1) ? h : 0.0);
}

/* Node weights with complex positions, for the complex-step derivative.  Same construction
 * as node_weights, with every step analytic in the positions: the edge frame (midpoint and
 * length) is formed from the complex offsets too, and the per-edge A comes from the normal
 * equations instead of the SVD route -- for a stencil of k >= 6 particles the minimum-norm
 * solution A = P^T y with (P P^T) y = b, for k < 6 (P of full column rank k: five particles
 * lie on one conic, so the six conditions cannot all hold) the least-squares solution
 * A = (P^T P)^-1 P^T b; both equal the pseudo-inverse solution P^+ b of the SVD route.  The
 * symmetric systems are factorised by a complex-symmetric Cholesky.  Topology is taken from
 * the real parts. */
static void csym_cholesky_solve(int m, cplx G[][6], cplx *rhs, cplx *x)
{
    cplx L[6][6], z[6];
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) L[r][c] = 0;
    for (int c = 0; c < m; ++c) {
        cplx acc = G[c][c];
        for (int j = 0; j < c; ++j) acc -= L[c][j] * L[c][j];
        L[c][c] = __builtin_csqrt(acc);
        for (int r = c + 1; r < m; ++r) {
            cplx a2 = G[r][c];
            for (int j = 0; j < c; ++j) a2 -= L[r][j] * L[c][j];
            L[r][c] = a2 / L[c][c];
        }
    }
    for (int r = 0; r < m; ++r) {
        cplx acc = rhs[r];
        for (int j = 0; j < r; ++j) acc -= L[r][j] * z[j];
        z[r] = acc / L[r][r];
    }
    for (int r = m - 1; r >= 0; --r) {
        cplx acc = z[r];
        for (int j = r + 1; j < m; ++j) acc -= L[j][r] * x[j];
        x[r] = acc / L[r][r];
    }
}

static void node_weights_cplx(const Geo *g, const NodeQ *Q, int I, int J, int shape,
                              int32_t kslot, int dim, double h, CSet *out)
{
    int nc = g->nc;
    double xq = (double)(I % nc) / nc, yq = (double)(J % nc) / nc;
    cplx d[3][2];
    for (int e = 0; e < 3; ++e)
        coffset(g, Q->w.p[Q->tri[e]].slot, xq, yq, kslot, dim, h, &d[e][0], &d[e][1]);
    cplx area2 = (d[1][0] - d[0][0]) * (d[2][1] - d[0][1]) - (d[1][1] - d[0][1]) * (d[2][0] - d[0][0]);
    cplx lam[3];
    lam[0] = (d[1][0] * d[2][1] - d[1][1] * d[2][0]) / area2;
    lam[1] = (d[2][0] * d[0][1] - d[2][1] * d[0][0]) / area2;
    lam[2] = (d[0][0] * d[1][1] - d[0][1] * d[1][0]) / area2;
    out->n = 0;
    for (int e = 0; e < 3; ++e) cset_add(out, Q->w.p[Q->tri[e]].slot, lam[e]);
    if (shape != 1) return;
    for (int e = 0; e < 3; ++e) {
        int f = (e + 1) % 3;
        int S[2 + 2 * OR_KSTAR];
        int k = edge_stencil(Q, e, S);
        cplx mx = 0.5 * (d[e][0] + d[f][0]), my = 0.5 * (d[e][1] + d[f][1]);
        cplx ex = d[e][0] - d[f][0], ey = d[e][1] - d[f][1];
        cplx s = __builtin_csqrt(ex * ex + ey * ey);
        cplx p[OR_KSTEN][6];
        for (int i = 0; i < k; ++i) {
            cplx dx, dy;
            coffset(g, Q->w.p[S[i]].slot, xq, yq, kslot, dim, h, &dx, &dy);
            cplx x = (dx - mx) / s, y = (dy - my) / s;
            p[i][0] = 1; p[i][1] = x; p[i][2] = y; p[i][3] = x * x; p[i][4] = x * y; p[i][5] = y * y;
        }
        cplx tx = ex / s, ty = ey / s;
        cplx b[6] = {0, 0, 0, -0.5 * tx * tx, -0.5 * tx * ty, -0.5 * ty * ty};
        cplx A[OR_KSTEN];
        if (k >= 6) {
            cplx M[6][6], y[6];
            for (int r = 0; r < 6; ++r)
                for (int c = 0; c < 6; ++c) {
                    M[r][c] = 0;
                    for (int i = 0; i < k; ++i) M[r][c] += p[i][r] * p[i][c];
                }
            csym_cholesky_solve(6, M, b, y);
            for (int i = 0; i < k; ++i) {
                A[i] = 0;
                for (int r = 0; r < 6; ++r) A[i] += p[i][r] * y[r];
            }
        } else {
            cplx Gm[6][6], rhs[6];
            for (int i = 0; i < k; ++i) {
                rhs[i] = 0;
                for (int r = 0; r < 6; ++r) rhs[i] += p[i][r] * b[r];
                for (int j = 0; j < k; ++j) {
                    Gm[i][j] = 0;
                    for (int r = 0; r < 6; ++r) Gm[i][j] += p[i][r] * p[j][r];
                }
            }
            csym_cholesky_solve(k, Gm, rhs, A);
        }
        cplx cf = 2.0 * lam[e] * lam[f];
        for (int i = 0; i < k; ++i) cset_add(out, Q->w.p[S[i]].slot, cf * A[i]);
    }
}

/* Derivatives of the weights of node (I, J) with respect to coordinate `dim` of original
 * particle m (complex step, h = 1e-30): writes dw[i] for the node's weight set as returned
 * by or_node_weights (same order). */
int or_node_weight_derivs(int n, int64_t N, const double *pos, const int32_t *cell_start,
                          const int32_t *perm, const uint32_t *qs, int I, int J, int shape,
                          int64_t m, int dim, int kmax, int32_t *idx, double *dw, int *count)
{
    Geo g = make_geo(n, N, pos, cell_start, perm, qs);
    NodeQ Q;
    memset(&Q, 0, sizeof(Q));
    WSet s;
    int st = node_weights(&g, I, J, shape, &s, &Q, NULL);
    if (st == OR_OK && s.n > kmax) st = OR_ERR_CAPACITY;
    if (st == OR_OK) {
        int32_t kslot = -1;
        for (int64_t q = 0; q < N; ++q)
            if (perm[q] == m) { kslot = (int32_t)q; break; }
        const double h = 1e-30;
        CSet cs_;
        node_weights_cplx(&g, &Q, I, J, shape, kslot, dim, h, &cs_);
        for (int i = 0; i < s.n; ++i) {
            idx[i] = perm[s.slot[i]];
            dw[i] = 0;
            for (int j = 0; j < cs_.n; ++j)
                if (cs_.slot[j] == s.slot[i]) dw[i] = __imag__ cs_.w[j] / h;
        }
        *count = s.n;
    }
    win_free(&Q.w);
    return st;
}

/* Adjoint of P2M for L with dL/dmesh = grad_mesh ([n*n, C], image entries included, each
 * stored entry treated as its own output):
 *   grad_vals[mu] = sum_i w_{i mu} g_i                          (transpose of the weights)
 *   grad_pos[kappa] = sum_i sum_c g_ic sum_mu vals_mu,c dw_{i mu}/dr_kappa   (complex step)
 * Nodes in [node_begin, node_end) only (the rest contribute nothing); serial, fixed order. */
int or_p2m_backward(int n, int64_t N, const double *pos, int C, const double *vals, int shape,
                    const double *grad_mesh, double *grad_vals, double *grad_pos,
                    int64_t node_begin, int64_t node_end)
{
    if (n < 3 || N < 3 || C < 1) return OR_ERR_ARG;
    int64_t ncell = (int64_t)(n - 1) * (n - 1);
    int32_t *cs = (int32_t *)xcalloc((size_t)ncell + 1, sizeof(int32_t));
    int32_t *perm = (int32_t *)xcalloc((size_t)N, sizeof(int32_t));
    uint32_t *qs = (uint32_t *)xcalloc((size_t)N * 2, sizeof(uint32_t));
    or_build_cells(n, N, pos, cs, perm, qs);
    Geo g = make_geo(n, N, pos, cs, perm, qs);
    for (int64_t i = 0; i < N * C; ++i) grad_vals[i] = 0;
    for (int64_t i = 0; i < N * 2; ++i) grad_pos[i] = 0;
    int64_t nn = (int64_t)n * n;
    if (node_end < 0 || node_end > nn) node_end = nn;
    if (node_begin < 0 || node_begin > node_end) {
        free(cs); free(perm); free(qs);
        return OR_ERR_ARG;
    }
    NodeQ Q;
    memset(&Q, 0, sizeof(Q));
    WSet s;
    CSet cs_;
    int err = OR_OK;
    const double h = 1e-30;
    for (int64_t node = node_begin; node < node_end && !err; ++node) {
        int J = (int)(node / n), I = (int)(node % n);
        const double *gb = grad_mesh + node * C;
        int any = 0;
        for (int c = 0; c < C; ++c) any |= gb[c] != 0.0;
        if (!any) continue;
        err = node_weights(&g, I, J, shape, &s, &Q, NULL);
        if (err) break;
        for (int i = 0; i < s.n; ++i)
            for (int c = 0; c < C; ++c) grad_vals[(int64_t)perm[s.slot[i]] * C + c] += s.w[i] * gb[c];
        for (int i = 0; i < s.n; ++i) {
            int32_t ks = s.slot[i];
            for (int dim = 0; dim < 2; ++dim) {
                node_weights_cplx(&g, &Q, I, J, shape, ks, dim, h, &cs_);
                double dv = 0;
                for (int j = 0; j < cs_.n; ++j) {
                    double dwj = __imag__ cs_.w[j] / h;
                    double gv = 0;
                    for (int c = 0; c < C; ++c) gv += gb[c] * vals[(int64_t)perm[cs_.slot[j]] * C + c];
                    dv += dwj * gv;
                }
                grad_pos[(int64_t)perm[ks] * 2 + dim] += dv;
            }
        }
    }
    win_free(&Q.w);
    free(cs); free(perm); free(qs);
    return err;
}

int or_abi_version(void) { return 1; }
