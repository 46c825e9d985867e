// internal.h -- declarations shared by the translation units of libpfem (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/pfem.h"
#include "common.cuh"

namespace pfem {

// Launch counter behind pfem_launch_count(); every kernel launch site calls count_launch().
void count_launch(unsigned k = 1);

// Multiprocessors of the current device (queried once per device), for grid sizes.
int num_sms();

// Byte offsets of the workspace regions (the status word always sits at offset 0).
struct WsLayout {
    size_t status, count, key, rank, scan, bwd, total;
};

WsLayout ws_layout(int n, int nb, long long N, int C);
WsLayout ws_layout_bins(long long nbins, long long N);
cudaError_t launch_sort_gather(long long nbins, long long N, const void *pos, pfem_dtype pos_t,
                               const int *key, int *rank, const int *cell_start, int *perm,
                               void *pos_sorted, uint32_t *q_sorted, cudaStream_t s);
size_t batch_plan_bytes(int P);
int batch_plan_build(int P, const pfem_batch_problem *probs, void *plan_dev, long long *N_total,
                     long long *bins_total, long long *nodes_total);
cudaError_t launch_batch_build_cells(const void *plan, long long Ntot, long long bins_total,
                                     const void *pos, pfem_dtype pos_t, int *cell_start, int *perm,
                                     void *pos_sorted, uint32_t *q_sorted, const WsLayout &L,
                                     void *ws, cudaStream_t s);
cudaError_t launch_batch_p2m(const void *plan, const void *pos_sorted, const uint32_t *q_sorted,
                             const int *cell_start, const int *perm, int C, const void *vals,
                             pfem_dtype val_t, pfem_shape shape, pfem_solve solve, void *mesh,
                             int shape_idx, int blocks, long long nodes_total, long long N_total,
                             void *ws, size_t ws_bytes, cudaStream_t s);
size_t batch_p2m_ws_bytes(long long nodes_total, long long N_total);
cudaError_t launch_batch_m2p(const void *plan, const void *pos, pfem_dtype pos_t, int C,
                             const void *mesh, void *vals, pfem_dtype val_t, int blocks,
                             cudaStream_t s);
size_t scan_scratch_ints(long long n);
cudaError_t scan_exclusive(const int *in, int *out, long long n, int *scratch, cudaStream_t s);

cudaError_t launch_build_cells(int nb, long long N, const void *pos, pfem_dtype pos_t,
                               int *cell_start, int *perm, void *pos_sorted, uint32_t *q_sorted,
                               const WsLayout &L, void *ws, cudaStream_t s);

struct GeoArgs {
    int n, nb;
    long long N;
    const void *pos_sorted;
    pfem_dtype pos_t;
    const uint32_t *q_sorted;
    const int *cell_start;
    int R0, rmax;
    float dmax;
    int rmax_far;               // search radius (bins) of the retry and fix passes
    int kcap;                   // star capacity (<= PFEM_KMAX)
    int walk_cap;               // visibility-walk steps
    int ucap;                   // distinct particles of one node in the fast pass (<= PFEM_UMAX)
    void *const *events = nullptr;  // stage events of the caller's context (cudaEvent_t), or null
    int nevents = 0;
    void *vals_event = nullptr;     // the context's values event (cudaEvent_t), or null
};

// Make stream s wait for the context's values event before a kernel that reads the values.
inline cudaError_t wait_values(const GeoArgs &g, cudaStream_t s)
{
    return g.vals_event ? cudaStreamWaitEvent(s, (cudaEvent_t)g.vals_event, 0) : cudaSuccess;
}

// Record stage event k of g on stream s (no-op without events).
inline void stage_event(const GeoArgs &g, int k, cudaStream_t s)
{
    if (g.events && k < g.nevents && g.events[k]) cudaEventRecord((cudaEvent_t)g.events[k], s);
}

struct StarTab;
struct Bins;
// Star table (startab.cuh): bytes for N particles, its layout from `base` (qcount: the queue
// counter), and the launches that fill it.
size_t star_tab_bytes(long long N);
unsigned next_tab_gen();
StarTab star_tab_layout(char *base, long long N, int *qcount);
cudaError_t launch_star_table(const Bins &B, int R0, int rmax_far, const StarTab &t,
                              DevStatus *st, cudaStream_t s);


cudaError_t launch_p2m(const GeoArgs &g, const int *perm, int C, const void *vals,
                       pfem_dtype val_t, pfem_shape shape, pfem_solve solve, void *out,
                       DevStatus *st, size_t ws_bytes, cudaStream_t s);
// Workspace bytes P2M uses for n*n nodes and N particles (fix-pass queue, node records, star
// table).
size_t p2m_ws_bytes(long long nodes, long long N);
cudaError_t launch_shape(const GeoArgs &g, pfem_shape shape, pfem_solve solve, int K, int *w_idx,
                         void *w, pfem_dtype w_t, DevStatus *st, size_t ws_bytes, cudaStream_t s);
cudaError_t launch_apply(int n, const int *perm, int C, const void *vals, pfem_dtype val_t,
                         const int *w_idx, const void *w, int K, pfem_dtype w_t, void *out,
                         cudaStream_t s);
cudaError_t launch_stars(const GeoArgs &g, int *nbrs, int *counts, DevStatus *st, cudaStream_t s);
size_t stars_ws_bytes(long long N);
cudaError_t launch_m2p_quadratic(int n, long long N, const void *pos, pfem_dtype pos_t, int C,
                                 const void *mesh, void *vals, pfem_dtype val_t, cudaStream_t s);
cudaError_t launch_m2p(int n, long long N, const void *pos, pfem_dtype pos_t, int C,
                       const void *mesh, void *vals, pfem_dtype val_t, cudaStream_t s);

cudaError_t launch_advect_midpoint(int n, long long N, const void *pos, pfem_dtype pos_t,
                                   const void *vel, double dt, void *out, cudaStream_t s);
size_t update_ws_bytes(long long nbins, long long N);
cudaError_t launch_update_cells(int nb, long long N, const void *pos, pfem_dtype pos_t,
                                const int *start_old, const int *perm_old, const uint32_t *q_old,
                                int *cell_start, int *perm, void *pos_sorted, uint32_t *q_sorted,
                                void *ws, cudaStream_t s);

struct BwdLayout {
    int K;   // entries per node written by the recompute kernel
    size_t e_slot, e_w, e_dpos, count, start, rank, order, scan, rec, tab, queue, total;   // rec: node records, tab: star table, queue: fix-pass nodes
};
BwdLayout bwd_layout(int n, long long N, int K);

cudaError_t launch_p2m_backward(const GeoArgs &g, const int *perm, int C, const void *vals,
                                pfem_dtype val_t, pfem_shape shape, pfem_solve solve,
                                bool checkpoint, const int *w_idx, const void *w, int Kw,
                                const void *grad_mesh, void *grad_vals, void *grad_pos,
                                const BwdLayout &L, void *ws, cudaStream_t s);
cudaError_t launch_m2p_backward(int n, int nb, long long N, const void *pos, pfem_dtype pos_t,
                                const int *cell_start, const int *perm, int C, const void *mesh,
                                const void *gv, pfem_dtype val_t, void *gm, void *gp,
                                cudaStream_t s);

}  // namespace pfem
