/*
 * pfem.h -- C ABI of the GB300 particle <-> fixed-mesh projection library (libpfem.so).
 *
 * The library implements, as CUDA kernels for sm_103a, the projection round trip of
 * Duque & Espanol, "Rapid convergence for simulations that project from particles onto a
 * fixed mesh" (arXiv 1610.05266), in 2D on the unit periodic square:
 *
 *   P2M  (Sec. 2.2, eq. p2m):  alpha_i  = sum_mu alpha_mu psi^p_mu(r_i)   at mesh nodes
 *   M2P  (Sec. 2.2, eq. m2p):  alpha_mu = sum_i  alpha_i  psi^m_i(r_mu)   at particles
 *
 * psi^p is either the linear finite-element shape function on the particles' Delaunay
 * triangulation (App. B, eqs. C0-C1) or the quadratically consistent shape function of
 * App. B eq. (phiquad), psi_mu = phi_mu + sum_{nu sigma} A_{mu nu sigma} phi_nu phi_sigma,
 * with A for each Delaunay edge the minimum-norm solution of eqs. (A0), (A1), (condquad)
 * over the edge's stencil (both endpoints and their Delaunay neighbours; App. A solves it
 * "by SVD with rank detection").  psi^m is linear FE on the fixed structured mesh.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Domain: unit periodic square.  Positions are (x, y) pairs, any real values with
 *    |x|,|y| < 2^20; they are taken modulo 1.
 *  - Mesh: n x n nodes including the stored periodic image row and column (n >= 9),
 *    spacing H = 1/(n-1).  Node (I, J) is at (I*H, J*H) and its C values are stored at
 *    mesh_vals[(J*n + I)*C + c].  Row/column n-1 hold copies of row/column 0.  Each cell is
 *    split along its (i,j)->(i+1,j+1) diagonal.
 *  - Topology (bins, Delaunay, point location) uses fixed-point coordinates
 *    q = round_half_even(x * 2^32) mod 2^32; Delaunay ties among cocircular particles are
 *    broken by perturbing lifted heights in the order of the key (qy << 32 | qx).
 *    Duplicate particles are rejected (PFEM_ERR_DEGENERATE).
 *  - Particle bins: an nb x nb grid, bin (bx, by) = ((qx*nb) >> 32, (qy*nb) >> 32), bin id
 *    by*nb + bx.  pfem_default_bins() picks nb for about 4 particles per bin.
 *  - Arrays are row-major and contiguous.  All device pointers are CUDA device (or managed)
 *    memory allocated by the caller; the library allocates nothing.  `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).  Every call is
 *    asynchronous on `stream`; host-detectable argument errors come back as the return
 *    code and launch nothing.
 *  - Errors found on the device (capacity, degeneracy, iteration caps) are recorded in the
 *    status word at the start of the workspace `ws`; pfem_read_status() synchronises the
 *    stream and returns it.  Kernels never trap and every loop is bounded.
 *  - Storage dtypes: positions PFEM_F64 or PFEM_F32; particle and mesh values PFEM_F64,
 *    PFEM_F32 or PFEM_BF16 (BF16 is storage only; arithmetic is FP32).  Arithmetic is FP64
 *    when values are PFEM_F64, FP32 otherwise; `solve` selects the precision of the 6x6
 *    moment systems independently.
 *  - Context: every compute entry point takes a `pfem_ctx *` first.  A context holds the
 *    options below (caps of the bounded loops, search radii, batch launch shapes) and the text
 *    of its last host-side error; NULL means the default options, with errors kept per host
 *    thread.  A context is plain host memory: it allocates nothing on the device, and calls
 *    with one context from several host threads must not overlap (its error text is shared).
 *    The paper has no counterpart of contexts or options.
 */
#ifndef PFEM_H
#define PFEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PFEM_OK = 0,
    PFEM_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported dtype combination */
    PFEM_ERR_CUDA = 2,          /* a CUDA launch or runtime call failed */
    PFEM_ERR_WORKSPACE = 3,     /* ws_bytes smaller than the matching *_workspace_size() */
    PFEM_ERR_CAPACITY = 4,      /* device: star > PFEM_KMAX, stencil or weight list overflow,
                                   search region exhausted */
    PFEM_ERR_DEGENERATE = 5,    /* device: duplicate particles or rank-deficient moments */
    PFEM_ERR_TIMEOUT = 6        /* device: a bounded loop hit its iteration cap */
} pfem_status;

typedef enum { PFEM_F64 = 0, PFEM_F32 = 1, PFEM_BF16 = 2 } pfem_dtype;
typedef enum { PFEM_SHAPE_LINEAR = 0, PFEM_SHAPE_QUADRATIC = 1 } pfem_shape;
typedef enum {
    PFEM_SOLVE_F64 = 0,         /* moment assembly and Cholesky in FP64 */
    PFEM_SOLVE_F32 = 1,         /* in FP32 after centring/scaling by the edge length */
    PFEM_SOLVE_F32_REFINED = 2, /* FP32 Cholesky + one refinement step, FP64 residual */
    PFEM_SOLVE_F32_REFINED_FF = 3 /* FP32 Cholesky + one refinement step, residual in float-float
                                   (pairs of FP32 numbers, ~48-bit significand): the same
                                   refinement without FP64 instructions */
} pfem_solve;
typedef enum { PFEM_BACKWARD_RECOMPUTE = 0, PFEM_BACKWARD_CHECKPOINT = 1 } pfem_backward_mode;

#define PFEM_KMAX 16        /* max Delaunay neighbours of one particle */
#define PFEM_KW_MAX 64      /* max weights per node in the explicit-weight form */
#define PFEM_UMAX 24        /* max distinct particles of one node in the fast pass */

/* Options of a context.  Zero in a field means its default. */
typedef struct {
    int32_t walk_max_steps;    /* steps of the visibility walk that locates a mesh node in the
                                  particles' Delaunay triangulation (default 64); a node that
                                  needs more records PFEM_ERR_TIMEOUT.  -1: no step allowed */
    int32_t star_capacity;     /* Delaunay neighbours kept per particle, 3..PFEM_KMAX (default
                                  PFEM_KMAX); a larger star records PFEM_ERR_CAPACITY */
    int32_t node_capacity;     /* distinct particles of one node in the fast pass, 3..PFEM_UMAX
                                  (default PFEM_UMAX); a node with more goes to the fix pass */
    int32_t search_radius_max; /* widest search, in bins, of the retry and fix passes that take
                                  the stars and nodes the first search radius could not certify
                                  (sparse regions, voids); default: a quarter of the torus.  A
                                  search that exhausts it records PFEM_ERR_CAPACITY */
    int32_t batch_tile_rows;   /* node rows (4, 8, 16) of a batched P2M work item (default 8) */
    int32_t batch_p2m_blocks;  /* blocks of the persistent batched P2M (default 8 per SM) */
    int32_t batch_m2p_blocks;  /* blocks of the batched M2P (default 16 per SM) */
    int32_t reserved[9];       /* zero */
} pfem_options;

typedef struct pfem_ctx pfem_ctx;

/* Fill *opt with the defaults (every field explicit). */
void pfem_options_default(pfem_options *opt);

/* Create a context with the given options (NULL = defaults); *ctx receives it.  Returns
 * PFEM_ERR_INVALID_ARG for an option out of range (nothing created). */
pfem_status pfem_create(pfem_ctx **ctx, const pfem_options *opt);

/* Destroy a context (NULL is ignored). */
void pfem_destroy(pfem_ctx *ctx);

/* The options of a context, defaults filled in (ctx NULL: the defaults). */
pfem_status pfem_get_options(const pfem_ctx *ctx, pfem_options *opt);

/* Text of the last host-side error of calls made with ctx (ctx NULL: of the calling thread's
 * calls made without a context), or "" after a call that succeeded.  The pointer stays valid
 * until the next call with the same context (or on the same thread). */
const char *pfem_last_error(const pfem_ctx *ctx);

/* Stage events for timing: events[0..count) are cudaEvent_t handles created by the caller
 * (count <= 8; 0 clears them).  Every later pfem_project_p2m with this context records them on
 * its stream at the boundaries of its stages when the star-table path runs: 0 before the fast
 * pass, 1 after the star table, 2 after the per-node geometry kernel, 3 after the solve kernel,
 * 4 after the fix pass (where one kernel locates the nodes and solves, 2 is recorded right
 * before it and 3 after it; the other paths record 0 and 4 only).  The caller reads the intervals
 * with cudaEventElapsedTime after synchronising.  Recording adds no work to the kernels. */
pfem_status pfem_set_stage_events(pfem_ctx *ctx, void *const *events, int32_t count);

/* An event (cudaEvent_t as void*) that pfem_project_p2m calls made with this context wait on
 * (cudaStreamWaitEvent on the call's stream) right before their first kernel that reads the
 * particle values -- after the star table (and the node records, where they are written) of the
 * quadratic path, at the start of the others; NULL (the default) clears it.  A caller can so copy the values on another
 * stream while the call works on the positions.  The event must have been recorded (or never
 * recorded: then the wait is a no-op) when the call is made. */
pfem_status pfem_set_values_event(pfem_ctx *ctx, void *event);

/* Version of this ABI. */
int pfem_abi_version(void);

/* Number of kernels this library has launched in this process (all devices, all streams);
 * lets a caller count the launches inside a timed region.  No paper counterpart. */
uint64_t pfem_launch_count(void);

/* Human-readable name of a status code. */
const char *pfem_status_string(pfem_status s);

/* Bins per side for N particles on a mesh of n nodes per side: about 4 particles per bin,
 * at least 8 bins per side. */
int32_t pfem_default_bins(int32_t n, int64_t N);

/* Bytes of workspace `ws` needed by the calls below for these sizes (>= 256); with n > 0 it
 * includes the fix-pass queue, node records and star table of pfem_project_p2m. */
size_t pfem_workspace_size(int32_t n, int32_t nb, int64_t N, int32_t C);

/* Status word recorded by device code in `ws` since the last reset; synchronises `stream`
 * (the only synchronising call of the library).  *status_host = pfem_status value,
 * *detail_host = index of the first failing node or particle (or -1). */
pfem_status pfem_read_status(const void *ws, int32_t *status_host, int64_t *detail_host,
                             void *stream);

/* Reset the device status word in `ws` to PFEM_OK (asynchronous). */
pfem_status pfem_reset_status(void *ws, void *stream);

/* pfem_read_status for a context: the same synchronising read, and a device error is also
 * described in the context's last-error text. */
pfem_status pfem_get_device_status(pfem_ctx *ctx, const void *ws, int32_t *status_host,
                                   int64_t *detail_host, void *stream);

/* a1-a2: canonicalise positions to fixed point and bin the particles with a stable
 * counting sort, slots ordered by (bin, original index).
 *   pos        [N,2] pos_t, original order (device)
 *   cell_start [nb*nb+1] int32 out: slots of bin b are cell_start[b] .. cell_start[b+1]-1
 *   perm       [N] int32 out: original index of the particle in each slot
 *   pos_sorted [N,2] pos_t out: pos[perm[s]]
 *   q_sorted   [N,2] uint32 out: fixed-point coordinates of pos_sorted
 *   ws         workspace of pfem_workspace_size(n, nb, N, C) bytes
 * No paper counterpart: the paper locates particles through CGAL (App. A). */
pfem_status pfem_build_cells(pfem_ctx *ctx, int32_t nb, int64_t N, const void *pos, pfem_dtype pos_t,
                             int32_t *cell_start, int32_t *perm, void *pos_sorted,
                             uint32_t *q_sorted, void *ws, size_t ws_bytes, void *stream);

/* The binning of pfem_build_cells (same outputs, bit for bit) without a workspace argument,
 * for callers that cannot allocate device memory where they need the bins -- e.g. a plug-in
 * called from a host application that owns every device allocation, or a real-time loop that
 * must not take the device synchronisation an allocation can imply.  The paper has no
 * counterpart.  Its scratch is a fixed array compiled into the library (36.0 MiB = 37,757,440
 * bytes), held on every GPU that loads it until the process exits; this call allocates nothing.
 * Limits: N <= 4,194,304 particles and nb*nb <= 1,048,576 bins, else PFEM_ERR_CAPACITY
 * (nothing launched).  The first call on a device looks up the scratch's device address (with
 * that device current) and caches it: make that first call before any stream capture.  The
 * cached address belongs to the device's primary context: after the host application destroys
 * that context (cudaDeviceReset), this entry point must not be called again in the process.  All
 * calls share the one scratch array and it keeps the last call's contents (the bin counters
 * are cleared at the start of every call): calls that overlap on the GPU -- on different
 * streams without ordering, or from different host threads -- race and must not be issued. */
pfem_status pfem_build_cells_noalloc(int32_t nb, int64_t N, const void *pos, pfem_dtype pos_t,
                                     int32_t *cell_start, int32_t *perm, void *pos_sorted,
                                     uint32_t *q_sorted, void *stream);

/* Delaunay stars (App. B: neighbours = particles joined by a Delaunay edge) of every
 * particle, counter-clockwise from its nearest neighbour, in slot indices: nbrs [N, PFEM_KMAX]
 * int32 (unused entries -1), counts [N] int32 (0 for a star that failed; its error is in the
 * status word).  This is the star table the quadratic projections build for themselves: one
 * thread per particle computes the convex hull of the particle's neighbours within two mean
 * spacings inverted about it, and the particles whose hull cannot be certified are searched
 * again over growing regions.  ws holds at least 256 + 4 N bytes (the retry queue). */
pfem_status pfem_delaunay_stars(pfem_ctx *ctx, int32_t nb, int64_t N, const uint32_t *q_sorted,
                                const int32_t *cell_start, int32_t *nbrs, int32_t *counts,
                                void *ws, size_t ws_bytes, void *stream);

/* Explicit P2M weights per node (eq. p2m with the chosen shape functions):
 * w_idx [n*n, K] int32 slot indices (-1 = unused) and w [n*n, K] weights (FP64 when
 * w_t == PFEM_F64, else FP32), so that alpha_i = sum_k w[i,k] alpha[slot w_idx[i,k]].
 * K <= PFEM_KW_MAX; a node with more distinct particles records PFEM_ERR_CAPACITY.
 * Used by the checkpointed backward and by pfem_project_p2m with given weights.
 * Quadratic shape functions: the workspace beyond its first 512 bytes holds a queue of the
 * nodes the fast solve cannot take (see pfem_project_p2m). */
pfem_status pfem_shape_quadratic(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                                 pfem_dtype pos_t, const uint32_t *q_sorted,
                                 const int32_t *cell_start, pfem_shape shape, pfem_solve solve,
                                 int32_t K, int32_t *w_idx, void *w, pfem_dtype w_t, void *ws,
                                 size_t ws_bytes, void *stream);

/* P2M (Sec. 2.2 eq. p2m) at all n*n nodes (image row/column included).
 *   vals      [N, C] val_t: if perm != NULL, vals are in ORIGINAL particle order and slot s
 *             reads vals[perm[s]]; if perm == NULL, vals are already in slot order
 *   w_idx, w  NULL => shape functions computed on the fly (fused); else the weights from
 *             pfem_shape_quadratic (K per node, dtype w_t) are applied
 *   mesh_vals [n, n, C] val_t out
 * C in 1..8.
 * Quadratic shape functions: each edge's coefficient system (App. B) is solved by a Cholesky
 * factorisation of its 6x6 moment matrix.  The call runs a fast pass over every node and a fix
 * pass over the nodes the fast pass queued: a node with an edge whose pivot falls below the
 * fast tolerance (rank deficient, e.g. a stencil of five particles, or too ill-conditioned for
 * the precision: 3e-4 of the trace in FP32, 1e-6 in FP64), with more than the context's
 * node_capacity distinct particles, or whose search ran out of its first region (a sparse
 * region or a void), is recomputed in FP64 with the minimum-norm least-squares solution by SVD
 * (App. A) and searches up to the context's search_radius_max.  Linear shape functions queue
 * only the last kind.  Workspace layout after the 256-byte status block: the fix-pass queue
 * from byte 512 (8 bytes per node; with ws_bytes < 520 there is no queue and such nodes record
 * PFEM_ERR_DEGENERATE or PFEM_ERR_CAPACITY), then, for the quadratic apply form, 136 bytes of
 * record per node and the star table (72 bytes per particle).  With room for them the fast
 * pass is the star table of every particle (see pfem_delaunay_stars) and one kernel that, per
 * node, locates it with the table, builds its particle set and solves the three edge systems;
 * the float-float solve (PFEM_SOLVE_F32_REFINED_FF) splits that kernel in two, a geometry
 * kernel writing the node records and a solve kernel reading them.  With less room, one kernel
 * searches every node's stars itself (same results, slower).  The workspace of pfem_workspace_size() has room for
 * everything. */
pfem_status pfem_project_p2m(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                             pfem_dtype pos_t, const uint32_t *q_sorted,
                             const int32_t *cell_start, const int32_t *perm, int32_t C,
                             const void *vals, pfem_dtype val_t, pfem_shape shape,
                             pfem_solve solve, const int32_t *w_idx, const void *w, int32_t K,
                             pfem_dtype w_t, void *mesh_vals, void *ws, size_t ws_bytes,
                             void *stream);

/* M2P (Sec. 2.2 eq. m2p) with linear FE on the structured mesh, per particle in the order
 * of `pos`:  vals [N, C] val_t out,  mesh_vals [n, n, C] val_t.  C in 1..8.  Needs no
 * workspace and records no device errors. */
pfem_status pfem_interp_m2p(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos, pfem_dtype pos_t,
                            int32_t C, const void *mesh_vals, void *vals, pfem_dtype val_t,
                            void *stream);

/* Bytes of workspace pfem_project_backward needs (its own workspace; K = weights per node of
 * the checkpointed weights, 0 in recompute mode).  Holds per-node entries [n*n, max(K,32)]
 * and a transposed index over the N particles. */
size_t pfem_backward_workspace_size(int32_t n, int64_t N, int32_t K);

/* M2P (Sec. 2.2 eq. m2p) with quadratically consistent MESH shape functions (App. B applied
 * to the fixed mesh; Table 1's projFEM6/projFEMq interpolate mesh -> particles with them):
 * w_i = lambda_i [i in T] + sum over T's edges (P,Q) of 2 lambda_P lambda_Q A_{i,(P,Q)}, where
 * each mesh edge's stencil is the closed neighbourhood of its endpoints (10 nodes of the
 * (i,j)->(i+1,j+1)-split mesh) and A is the minimum-norm solution of eqs. A0, A1, condquad;
 * on the uniform mesh A depends only on the edge direction and is computed once.  Values
 * are read at the unique nodes (I mod (n-1), J mod (n-1)).  FP64 (FP64 positions), FP32 or
 * BF16 storage (FP32 positions).  No workspace, no device errors. */
pfem_status pfem_interp_m2p_quadratic(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos, pfem_dtype pos_t,
                                      int32_t C, const void *mesh_vals, void *vals,
                                      pfem_dtype val_t, void *stream);

/* Adjoint of P2M with respect to particle values and positions, for an upstream gradient
 * grad_mesh [n, n, C] (each stored entry, image copies included, is its own output):
 *   grad_vals [N, C] out (original order when perm != NULL, slot order otherwise)
 *   grad_pos  [N, 2] out, same order; NULL skips the position gradient
 * Topology is held fixed.  mode RECOMPUTE rebuilds the shape functions; mode CHECKPOINT
 * reads w_idx/w from pfem_shape_quadratic for the value gradient (positions are always
 * recomputed).  Deterministic: per-node entries, then a per-particle gather through a stable
 * counting sort (no atomics on values).  Values FP32 (solve F32 or F64) or FP64 (solve F64);
 * ws is a separate workspace of pfem_backward_workspace_size() bytes whose status word records
 * device errors.  A node with more than 32 distinct particles records PFEM_ERR_CAPACITY. */
pfem_status pfem_project_backward(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N, const void *pos_sorted,
                                  pfem_dtype pos_t, const uint32_t *q_sorted,
                                  const int32_t *cell_start, const int32_t *perm, int32_t C,
                                  const void *vals, pfem_dtype val_t, pfem_shape shape,
                                  pfem_solve solve, pfem_backward_mode mode,
                                  const int32_t *w_idx, const void *w, int32_t K,
                                  pfem_dtype w_t, const void *grad_mesh, void *grad_vals,
                                  void *grad_pos, void *ws, size_t ws_bytes, void *stream);

/* Adjoint of M2P for an upstream gradient grad_vals [N, C] (order of pos):
 *   grad_mesh [n, n, C] out: into the stored entry each forward read used
 *   grad_pos  [N, 2] out (NULL skips): grad_vals . gradient of the linear FE field
 * Deterministic: a per-node gather over the bins' particles (bins must be the
 * pfem_build_cells output for the same positions).  FP32 or FP64 values. */
pfem_status pfem_interp_m2p_backward(pfem_ctx *ctx, int32_t n, int32_t nb, int64_t N, const void *pos,
                                     pfem_dtype pos_t, const int32_t *cell_start,
                                     const int32_t *perm, int32_t C, const void *mesh_vals,
                                     const void *grad_vals, pfem_dtype val_t, void *grad_mesh,
                                     void *grad_pos, void *stream);

/* ------------------------------------------------------------------ the projection loop
 * Sec. 3.1 runs, on Zalesak's disk, a loop whose every step projects the field mesh ->
 * particles (M2P), moves the particles one step with the midpoint velocity, rebuilds the
 * particle shape functions and projects particles -> mesh (P2M).  These two calls are the
 * steps between the projections. */

/* Midpoint move (the scheme of Sec. 3.2): r_half = r + dt/2 u(r), r_new = r + dt u(r_half), with
 * u interpolated from the mesh velocity field mesh_vel [n, n, 2] (pos_t, same layout as M2P's
 * mesh values) by linear FE on the structured mesh (eq. m2p).  pos [N, 2] in any order,
 * pos_out [N, 2] in the same order, wrapped into [0, 1).  No workspace, no device errors. */
pfem_status pfem_advect_midpoint(pfem_ctx *ctx, int32_t n, int64_t N, const void *pos,
                                 pfem_dtype pos_t, const void *mesh_vel, double dt, void *pos_out,
                                 void *stream);

/* Bytes of workspace pfem_update_cells needs. */
size_t pfem_update_workspace_size(int32_t nb, int64_t N);

/* Re-bin particles that moved since the binning (cell_start_old, perm_old, q_sorted_old) of
 * pfem_build_cells or of an earlier call: pos [N, 2] are the new positions in original order;
 * the outputs are exactly those of pfem_build_cells(pos) provided every particle's new bin is
 * its old bin or one of the eight around it on the torus.  The new bins are filled from the
 * old ones without atomics: the particles that end in bin b come from the 3 x 3 old bins around
 * b, each in original-index order, so a particle's slot is the start of b plus the number of
 * those particles with a smaller original index.  A particle that moved further records
 * PFEM_ERR_CAPACITY in the status word of ws (detail: its original index) and the outputs are
 * then not valid: call pfem_build_cells.  The new arrays must not alias the old ones.  No paper
 * counterpart (the paper rebuilds a global triangulation, App. A). */
pfem_status pfem_update_cells(pfem_ctx *ctx, int32_t nb, int64_t N, const void *pos,
                              pfem_dtype pos_t, const int32_t *cell_start_old,
                              const int32_t *perm_old, const uint32_t *q_sorted_old,
                              int32_t *cell_start, int32_t *perm, void *pos_sorted,
                              uint32_t *q_sorted, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ batches
 * Many independent problems (their own mesh size, particle count and bins) processed in one
 * launch per stage.  The caller concatenates the problems: particles of problem p occupy rows
 * [poff_p, poff_p + N_p) of the particle arrays (pos, vals, pos_sorted, q_sorted, perm) in
 * problem order, its bins a contiguous range of one cell_start array and its n_p^2 nodes a
 * contiguous range of one mesh array; pfem_batch_plan_init reports the totals.  After
 * pfem_batch_build_cells, cell_start holds global slot indices and perm global particle
 * indices.  No paper counterpart (the paper runs one problem at a time). */
typedef struct {
    int32_t n;      /* mesh nodes per side (image row/column included), >= 9 */
    int32_t nb;     /* bins per side, >= 8 (pfem_default_bins) */
    int64_t N;      /* particles, >= 3 */
} pfem_batch_problem;

/* Bytes of the device plan for P problems. */
size_t pfem_batch_plan_size(int32_t P);

/* Build the plan (descriptors, search radii, work-item prefix tables) from P host
 * descriptors and copy it to `plan` (device memory of pfem_batch_plan_size(P) bytes); this
 * call synchronises.  totals[0..2] = total particles, total bins, total nodes. */
pfem_status pfem_batch_plan_init(pfem_ctx *ctx, int32_t P, const pfem_batch_problem *problems, void *plan,
                                 int64_t *totals);

/* Workspace bytes of pfem_batch_build_cells / pfem_batch_project_p2m for the totals of
 * pfem_batch_plan_init (nodes_total = 0: binning only). */
size_t pfem_batch_workspace_size(int64_t N_total, int64_t bins_total, int64_t nodes_total);

/* Binning of every problem at once (a1-a2 on the concatenated layout). */
pfem_status pfem_batch_build_cells(pfem_ctx *ctx, const void *plan, int64_t N_total, int64_t bins_total,
                                   const void *pos, pfem_dtype pos_t, int32_t *cell_start,
                                   int32_t *perm, void *pos_sorted, uint32_t *q_sorted, void *ws,
                                   size_t ws_bytes, void *stream);

/* P2M of every problem in one persistent launch: `blocks` blocks of 16 x tile_rows threads
 * (tile_rows 4, 8 or 16; 0 takes the context's batch_tile_rows, blocks 0 its
 * batch_p2m_blocks) pull (problem, 16 x tile_rows node tile) items from a counter in ws.
 * Values FP32 (FP32 positions) or FP64 (FP64 positions, FP64 solve).  nodes_total and N_total
 * must be totals[2] and totals[0] of the pfem_batch_plan_init call that built `plan`; the
 * workspace (pfem_batch_workspace_size with those totals) holds, after its 256-byte status
 * block, the fix-pass queue (8 bytes per node), the per-node records and the star table.
 * Quadratic shape functions then run as for one problem: the star table of every problem, a
 * persistent kernel that writes each node's record, a kernel that solves the edge systems,
 * and the fix pass over the queued nodes (FP64, SVD solve, widest search radius).  The
 * kernels compare the totals with the plan's own before writing anything and record
 * PFEM_ERR_INVALID_ARG (detail -1) when they differ.  With a smaller workspace (at least 256
 * bytes plus the queue) every node runs a fused per-node kernel; linear shape functions always
 * do.  Device errors carry batch-wide node (or particle) indices. */
pfem_status pfem_batch_project_p2m(pfem_ctx *ctx, const void *plan, int64_t nodes_total,
                                   int64_t N_total, const void *pos_sorted, pfem_dtype pos_t,
                                   const uint32_t *q_sorted, const int32_t *cell_start,
                                   const int32_t *perm, int32_t C, const void *vals,
                                   pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                   void *mesh_vals, int32_t tile_rows, int32_t blocks, void *ws,
                                   size_t ws_bytes, void *stream);

/* M2P of every problem in one launch of `blocks` blocks (0: the context's batch_m2p_blocks)
 * over 4096-particle chunks. */
pfem_status pfem_batch_interp_m2p(pfem_ctx *ctx, const void *plan, const void *pos, pfem_dtype pos_t, int32_t C,
                                  const void *mesh_vals, void *vals, pfem_dtype val_t,
                                  int32_t blocks, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PFEM_H */
