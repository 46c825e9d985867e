"""Python binding of the C ABI (one function per entry point, same names) plus a small
buffer-owning helper.  Only argument marshalling happens here: every step of the path runs
in libpfem's CUDA kernels; torch only provides device memory and the stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional, Tuple

import torch

from . import _lib as L
from ._lib import (PFEM_BACKWARD_CHECKPOINT, PFEM_BACKWARD_RECOMPUTE, PFEM_F32, PFEM_F64,  # noqa: F401
                   PFEM_KMAX, PFEM_KW_MAX, PFEM_SHAPE_LINEAR, PFEM_SHAPE_QUADRATIC,
                   PFEM_SOLVE_F32, PFEM_SOLVE_F32_REFINED, PFEM_SOLVE_F32_REFINED_FF,
                   PFEM_SOLVE_F64, PfemError, check,
                   dtype_code, ptr, stream_ptr)


def pfem_abi_version() -> int:
    return L.load().pfem_abi_version()


def pfem_launch_count() -> int:
    return int(L.load().pfem_launch_count())


class Context:
    """A pfem_ctx: options of the bounded searches and loops, and the last host-side error.
    Keyword arguments are pfem_options fields (walk_max_steps, star_capacity, node_capacity,
    search_radius_max, batch_tile_rows, batch_p2m_blocks, batch_m2p_blocks); zero or missing
    fields take their defaults."""

    def __init__(self, **options):
        lib = L.load()
        opts = L.Options(**options)
        h = ctypes.c_void_p()
        check(lib.pfem_create(ctypes.byref(h), ctypes.byref(opts)), "pfem_create")
        self.handle = h
        self._lib = lib

    def options(self) -> dict:
        o = L.Options()
        check(self._lib.pfem_get_options(self.handle, ctypes.byref(o)), "pfem_get_options", self)
        return {name: getattr(o, name) for name, _ in L.Options._fields_ if name != "reserved"}

    def last_error(self) -> str:
        return pfem_last_error(self)

    def set_stage_events(self, events):
        """torch.cuda.Event objects (created with enable_timing=True) recorded by later P2M calls
        at their stage boundaries (pfem_set_stage_events); [] clears them."""
        for e in events:
            if not e.cuda_event:
                e.record()                   # materialise the CUDA event handle
        arr = (ctypes.c_void_p * max(1, len(events)))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        check(self._lib.pfem_set_stage_events(self.handle, ctypes.cast(arr, ctypes.c_void_p), len(events)),
              "pfem_set_stage_events", self)
        self._events = list(events)

    def set_values_event(self, event):
        """A torch.cuda.Event that later P2M calls wait on before their first kernel that reads
        the particle values (pfem_set_values_event); None clears it."""
        if event is not None and not event.cuda_event:
            event.record()
        h = ctypes.c_void_p(event.cuda_event) if event is not None else None
        check(self._lib.pfem_set_values_event(self.handle, h), "pfem_set_values_event", self)
        self._values_event = event

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self._lib.pfem_destroy(h)
            self.handle = None


def pfem_last_error(ctx: Optional[Context] = None) -> str:
    t = L.load().pfem_last_error(L.ctx_ptr(ctx))
    return t.decode() if t else ""


def pfem_default_bins(n: int, N: int) -> int:
    return int(L.load().pfem_default_bins(n, N))


def pfem_workspace_size(n: int, nb: int, N: int, C: int) -> int:
    return int(L.load().pfem_workspace_size(n, nb, N, C))


def pfem_read_status(ws: torch.Tensor, stream=None) -> Tuple[int, int]:
    code, detail = ctypes.c_int32(0), ctypes.c_int64(0)
    check(L.load().pfem_read_status(ptr(ws), ctypes.byref(code), ctypes.byref(detail),
                                    stream_ptr(stream)), "pfem_read_status")
    return code.value, detail.value


def pfem_get_device_status(ws: torch.Tensor, stream=None, ctx=None) -> Tuple[int, int]:
    code, detail = ctypes.c_int32(0), ctypes.c_int64(0)
    check(L.load().pfem_get_device_status(L.ctx_ptr(ctx), ptr(ws), ctypes.byref(code),
                                          ctypes.byref(detail), stream_ptr(stream)),
          "pfem_get_device_status", ctx)
    return code.value, detail.value


def pfem_reset_status(ws: torch.Tensor, stream=None):
    check(L.load().pfem_reset_status(ptr(ws), stream_ptr(stream)), "pfem_reset_status")


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def pfem_build_cells(nb, N, pos, cell_start, perm, pos_sorted, q_sorted, ws, stream=None,
                     ctx=None):
    check(L.load().pfem_build_cells(L.ctx_ptr(ctx), nb, N, ptr(pos), dtype_code(pos.dtype),
                                    ptr(cell_start), ptr(perm), ptr(pos_sorted), ptr(q_sorted),
                                    ptr(ws), _nbytes(ws), stream_ptr(stream)),
          "pfem_build_cells", ctx)


def pfem_build_cells_noalloc(nb, N, pos, cell_start, perm, pos_sorted, q_sorted, stream=None):
    """pfem_build_cells without a workspace (scratch compiled into the library; see pfem.h)."""
    check(L.load().pfem_build_cells_noalloc(nb, N, ptr(pos), dtype_code(pos.dtype), ptr(cell_start),
                                            ptr(perm), ptr(pos_sorted), ptr(q_sorted),
                                            stream_ptr(stream)), "pfem_build_cells_noalloc")


def pfem_delaunay_stars(nb, N, q_sorted, cell_start, nbrs, counts, ws, stream=None, ctx=None):
    check(L.load().pfem_delaunay_stars(L.ctx_ptr(ctx), nb, N, ptr(q_sorted), ptr(cell_start),
                                       ptr(nbrs), ptr(counts), ptr(ws), _nbytes(ws),
                                       stream_ptr(stream)), "pfem_delaunay_stars", ctx)


def pfem_shape_quadratic(n, nb, N, pos_sorted, q_sorted, cell_start, shape, solve, K, w_idx, w,
                         ws, stream=None, ctx=None):
    check(L.load().pfem_shape_quadratic(L.ctx_ptr(ctx), n, nb, N, ptr(pos_sorted),
                                        dtype_code(pos_sorted.dtype), ptr(q_sorted),
                                        ptr(cell_start), shape, solve, K, ptr(w_idx), ptr(w),
                                        dtype_code(w.dtype), ptr(ws), _nbytes(ws),
                                        stream_ptr(stream)), "pfem_shape_quadratic", ctx)


def pfem_project_p2m(n, nb, N, pos_sorted, q_sorted, cell_start, perm, C, vals, shape, solve,
                     w_idx, w, K, mesh_vals, ws, stream=None, ctx=None):
    w_t = dtype_code(w.dtype) if w is not None else PFEM_F32
    check(L.load().pfem_project_p2m(L.ctx_ptr(ctx), n, nb, N, ptr(pos_sorted),
                                    dtype_code(pos_sorted.dtype), ptr(q_sorted), ptr(cell_start),
                                    ptr(perm), C, ptr(vals), dtype_code(vals.dtype), shape, solve,
                                    ptr(w_idx), ptr(w), K, w_t, ptr(mesh_vals), ptr(ws),
                                    _nbytes(ws), stream_ptr(stream)), "pfem_project_p2m", ctx)


def pfem_interp_m2p(n, N, pos, C, mesh_vals, vals, stream=None, ctx=None):
    check(L.load().pfem_interp_m2p(L.ctx_ptr(ctx), n, N, ptr(pos), dtype_code(pos.dtype), C,
                                   ptr(mesh_vals), ptr(vals), dtype_code(vals.dtype),
                                   stream_ptr(stream)), "pfem_interp_m2p", ctx)


def pfem_backward_workspace_size(n: int, N: int, K: int) -> int:
    return int(L.load().pfem_backward_workspace_size(n, N, K))


def pfem_interp_m2p_quadratic(n, N, pos, C, mesh_vals, vals, stream=None, ctx=None):
    check(L.load().pfem_interp_m2p_quadratic(L.ctx_ptr(ctx), n, N, ptr(pos), dtype_code(pos.dtype),
                                             C, ptr(mesh_vals), ptr(vals), dtype_code(vals.dtype),
                                             stream_ptr(stream)), "pfem_interp_m2p_quadratic", ctx)


def pfem_project_backward(n, nb, N, pos_sorted, q_sorted, cell_start, perm, C, vals, shape,
                          solve, mode, w_idx, w, K, grad_mesh, grad_vals, grad_pos, ws,
                          stream=None, ctx=None):
    w_t = dtype_code(w.dtype) if w is not None else PFEM_F32
    check(L.load().pfem_project_backward(L.ctx_ptr(ctx), n, nb, N, ptr(pos_sorted),
                                         dtype_code(pos_sorted.dtype), ptr(q_sorted),
                                         ptr(cell_start), ptr(perm), C, ptr(vals),
                                         dtype_code(vals.dtype), shape, solve, mode, ptr(w_idx),
                                         ptr(w), K, w_t, ptr(grad_mesh), ptr(grad_vals),
                                         ptr(grad_pos), ptr(ws), _nbytes(ws), stream_ptr(stream)),
          "pfem_project_backward", ctx)


def pfem_interp_m2p_backward(n, nb, N, pos, cell_start, perm, C, mesh_vals, grad_vals, grad_mesh,
                             grad_pos, stream=None, ctx=None):
    check(L.load().pfem_interp_m2p_backward(L.ctx_ptr(ctx), n, nb, N, ptr(pos),
                                            dtype_code(pos.dtype), ptr(cell_start), ptr(perm), C,
                                            ptr(mesh_vals), ptr(grad_vals),
                                            dtype_code(grad_vals.dtype), ptr(grad_mesh),
                                            ptr(grad_pos), stream_ptr(stream)),
          "pfem_interp_m2p_backward", ctx)


def pfem_advect_midpoint(n, N, pos, mesh_vel, dt, pos_out, stream=None, ctx=None):
    check(L.load().pfem_advect_midpoint(L.ctx_ptr(ctx), n, N, ptr(pos), dtype_code(pos.dtype),
                                        ptr(mesh_vel), float(dt), ptr(pos_out), stream_ptr(stream)),
          "pfem_advect_midpoint", ctx)


def pfem_update_workspace_size(nb: int, N: int) -> int:
    return int(L.load().pfem_update_workspace_size(nb, N))


def pfem_update_cells(nb, N, pos, cell_start_old, perm_old, q_sorted_old, cell_start, perm,
                      pos_sorted, q_sorted, ws, stream=None, ctx=None):
    check(L.load().pfem_update_cells(L.ctx_ptr(ctx), nb, N, ptr(pos), dtype_code(pos.dtype),
                                     ptr(cell_start_old), ptr(perm_old), ptr(q_sorted_old),
                                     ptr(cell_start), ptr(perm), ptr(pos_sorted), ptr(q_sorted),
                                     ptr(ws), _nbytes(ws), stream_ptr(stream)),
          "pfem_update_cells", ctx)


def pfem_batch_plan_size(P: int) -> int:
    return int(L.load().pfem_batch_plan_size(P))


def pfem_batch_plan_init(problems, plan: torch.Tensor, ctx=None):
    """problems: list of (n, nb, N).  Returns (N_total, bins_total, nodes_total)."""
    arr = (L.BatchProblem * len(problems))(*[L.BatchProblem(n, nb, N) for n, nb, N in problems])
    tot = (ctypes.c_int64 * 3)()
    check(L.load().pfem_batch_plan_init(L.ctx_ptr(ctx), len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                        ptr(plan), ctypes.cast(tot, ctypes.POINTER(ctypes.c_int64))),
          "pfem_batch_plan_init", ctx)
    return int(tot[0]), int(tot[1]), int(tot[2])


def pfem_batch_workspace_size(N_total: int, bins_total: int, nodes_total: int = 0) -> int:
    return int(L.load().pfem_batch_workspace_size(N_total, bins_total, nodes_total))


def pfem_batch_build_cells(plan, N_total, bins_total, pos, cell_start, perm, pos_sorted, q_sorted,
                           ws, stream=None, ctx=None):
    check(L.load().pfem_batch_build_cells(L.ctx_ptr(ctx), ptr(plan), N_total, bins_total, ptr(pos),
                                          dtype_code(pos.dtype), ptr(cell_start), ptr(perm),
                                          ptr(pos_sorted), ptr(q_sorted), ptr(ws), _nbytes(ws),
                                          stream_ptr(stream)), "pfem_batch_build_cells", ctx)


def pfem_batch_project_p2m(plan, nodes_total, N_total, pos_sorted, q_sorted, cell_start, perm, C,
                           vals, shape, solve, mesh_vals, tile_rows, blocks, ws, stream=None,
                           ctx=None):
    check(L.load().pfem_batch_project_p2m(L.ctx_ptr(ctx), ptr(plan), nodes_total, N_total,
                                          ptr(pos_sorted), dtype_code(pos_sorted.dtype),
                                          ptr(q_sorted), ptr(cell_start), ptr(perm), C, ptr(vals),
                                          dtype_code(vals.dtype), shape, solve, ptr(mesh_vals),
                                          tile_rows, blocks, ptr(ws), _nbytes(ws),
                                          stream_ptr(stream)), "pfem_batch_project_p2m", ctx)


def pfem_batch_interp_m2p(plan, pos, C, mesh_vals, vals, blocks, stream=None, ctx=None):
    check(L.load().pfem_batch_interp_m2p(L.ctx_ptr(ctx), ptr(plan), ptr(pos), dtype_code(pos.dtype),
                                         C, ptr(mesh_vals), ptr(vals), dtype_code(vals.dtype),
                                         blocks, stream_ptr(stream)), "pfem_batch_interp_m2p", ctx)


@dataclass
class Cells:
    """Device buffers of one binned particle set (output of pfem_build_cells)."""
    n: int
    nb: int
    N: int
    cell_start: torch.Tensor
    perm: torch.Tensor
    pos_sorted: torch.Tensor
    q_sorted: torch.Tensor
    ws: torch.Tensor


class Projector:
    """Owns the device buffers for one problem size and runs the round trip through the ABI."""

    def __init__(self, n: int, N: int, C: int = 1, nb: Optional[int] = None,
                 pos_dtype: torch.dtype = torch.float64, device="cuda",
                 ctx: Optional[Context] = None):
        self.n, self.N, self.C = n, N, C
        self.ctx = ctx
        self.nb = nb if nb is not None else pfem_default_bins(n, N)
        self.device = torch.device(device)
        ws_bytes = pfem_workspace_size(n, self.nb, N, C)
        dev = self.device
        self.cells = Cells(
            n, self.nb, N,
            torch.empty(self.nb * self.nb + 1, dtype=torch.int32, device=dev),
            torch.empty(max(N, 1), dtype=torch.int32, device=dev),
            torch.empty((max(N, 1), 2), dtype=pos_dtype, device=dev),
            torch.empty((max(N, 1), 2), dtype=torch.int32, device=dev),
            torch.zeros((ws_bytes + 15) // 16 * 2, dtype=torch.float64, device=dev),
        )

    @property
    def ws(self) -> torch.Tensor:
        return self.cells.ws

    def build(self, pos: torch.Tensor, stream=None):
        c = self.cells
        pfem_build_cells(self.nb, self.N, pos, c.cell_start, c.perm, c.pos_sorted, c.q_sorted,
                         c.ws, stream, ctx=self.ctx)
        return c

    def p2m(self, vals: torch.Tensor, shape=PFEM_SHAPE_QUADRATIC, solve=None, out=None,
            sorted_vals: bool = False, weights=None, stream=None) -> torch.Tensor:
        c = self.cells
        C = vals.shape[1]
        if solve is None:
            solve = PFEM_SOLVE_F64 if vals.dtype == torch.float64 else PFEM_SOLVE_F32
        if out is None:
            out = torch.empty((self.n, self.n, C), dtype=vals.dtype, device=vals.device)
        w_idx, w = (weights if weights is not None else (None, None))
        K = w_idx.shape[1] if w_idx is not None else 0
        pfem_project_p2m(self.n, self.nb, self.N, c.pos_sorted, c.q_sorted, c.cell_start,
                         None if sorted_vals else c.perm, C, vals, shape, solve, w_idx, w, K, out,
                         c.ws, stream, ctx=self.ctx)
        return out

    def shape_weights(self, shape=PFEM_SHAPE_QUADRATIC, solve=None, K: int = 32,
                      w_dtype=None, stream=None):
        c = self.cells
        w_dtype = w_dtype or c.pos_sorted.dtype
        if solve is None:
            solve = PFEM_SOLVE_F64 if w_dtype == torch.float64 else PFEM_SOLVE_F32
        nn = self.n * self.n
        w_idx = torch.empty((nn, K), dtype=torch.int32, device=self.device)
        w = torch.empty((nn, K), dtype=w_dtype, device=self.device)
        pfem_shape_quadratic(self.n, self.nb, self.N, c.pos_sorted, c.q_sorted, c.cell_start,
                             shape, solve, K, w_idx, w, c.ws, stream, ctx=self.ctx)
        return w_idx, w

    def stars(self, stream=None):
        c = self.cells
        nbrs = torch.empty((self.N, PFEM_KMAX), dtype=torch.int32, device=self.device)
        counts = torch.empty(self.N, dtype=torch.int32, device=self.device)
        pfem_delaunay_stars(self.nb, self.N, c.q_sorted, c.cell_start, nbrs, counts, c.ws, stream, ctx=self.ctx)
        return nbrs, counts

    def m2p(self, pos: torch.Tensor, mesh: torch.Tensor, out=None, shape=PFEM_SHAPE_LINEAR,
            stream=None) -> torch.Tensor:
        """M2P with linear FE (default) or quadratically consistent mesh shape functions."""
        C = mesh.shape[-1]
        if out is None:
            out = torch.empty((pos.shape[0], C), dtype=mesh.dtype, device=mesh.device)
        if shape == PFEM_SHAPE_QUADRATIC:
            pfem_interp_m2p_quadratic(self.n, pos.shape[0], pos, C, mesh, out, stream, ctx=self.ctx)
        else:
            pfem_interp_m2p(self.n, pos.shape[0], pos, C, mesh, out, stream, ctx=self.ctx)
        return out

    def backward(self, vals: torch.Tensor, grad_mesh: torch.Tensor, shape=PFEM_SHAPE_QUADRATIC,
                 solve=None, weights=None, want_pos: bool = True, sorted_vals: bool = False,
                 stream=None):
        """Adjoint of p2m: (grad_vals [N,C], grad_pos [N,2] or None), same order as vals.
        With `weights` (from shape_weights) the value gradient uses them (checkpoint mode)."""
        c = self.cells
        C = vals.shape[1]
        if solve is None:
            solve = PFEM_SOLVE_F64 if vals.dtype == torch.float64 else PFEM_SOLVE_F32
        w_idx, w = weights if weights is not None else (None, None)
        K = w_idx.shape[1] if w_idx is not None else 0
        mode = PFEM_BACKWARD_CHECKPOINT if weights is not None else PFEM_BACKWARD_RECOMPUTE
        nbytes = pfem_backward_workspace_size(self.n, self.N, K)
        if getattr(self, "_bws", None) is None or self._bws.numel() * 8 < nbytes:
            self._bws = torch.zeros((nbytes + 7) // 8, dtype=torch.float64, device=self.device)
        else:
            pfem_reset_status(self._bws, stream)
        gv = torch.empty_like(vals)
        gp = torch.empty((self.N, 2), dtype=vals.dtype, device=self.device) if want_pos else None
        pfem_project_backward(self.n, self.nb, self.N, c.pos_sorted, c.q_sorted, c.cell_start,
                              None if sorted_vals else c.perm, C, vals, shape, solve, mode, w_idx,
                              w, K, grad_mesh.contiguous(), gv, gp, self._bws, stream, ctx=self.ctx)
        return gv, gp

    def backward_status(self, stream=None) -> Tuple[int, int]:
        return pfem_get_device_status(self._bws, stream, ctx=self.ctx)

    def m2p_backward(self, pos: torch.Tensor, mesh: torch.Tensor, grad_vals: torch.Tensor,
                     want_pos: bool = True, stream=None):
        """Adjoint of m2p for positions binned by the last build(pos)."""
        c = self.cells
        C = mesh.shape[-1]
        gm = torch.empty_like(mesh)
        gp = torch.empty((pos.shape[0], 2), dtype=mesh.dtype, device=self.device) if want_pos else None
        pfem_interp_m2p_backward(self.n, self.nb, pos.shape[0], pos, c.cell_start, c.perm, C,
                                 mesh.contiguous(), grad_vals.contiguous(), gm, gp, stream, ctx=self.ctx)
        return gm, gp

    def advect(self, pos: torch.Tensor, mesh_vel: torch.Tensor, dt: float, out=None,
               stream=None) -> torch.Tensor:
        """Midpoint move of pos (any order) in the mesh velocity field mesh_vel [n, n, 2]."""
        if out is None:
            out = torch.empty_like(pos)
        pfem_advect_midpoint(self.n, pos.shape[0], pos, mesh_vel.contiguous(), dt, out, stream,
                             ctx=self.ctx)
        return out

    def update(self, pos: torch.Tensor, stream=None):
        """Re-bin after a move of at most one bin per particle (pfem_update_cells): the new
        binning goes to a second set of buffers, which then becomes the current one."""
        c = self.cells
        alt = getattr(self, "_alt", None)
        if alt is None:
            dev = self.device
            alt = Cells(c.n, c.nb, c.N, torch.empty_like(c.cell_start), torch.empty_like(c.perm),
                        torch.empty_like(c.pos_sorted), torch.empty_like(c.q_sorted), c.ws)
        pfem_update_cells(self.nb, self.N, pos, c.cell_start, c.perm, c.q_sorted, alt.cell_start,
                          alt.perm, alt.pos_sorted, alt.q_sorted, c.ws, stream, ctx=self.ctx)
        self._alt, self.cells = c, alt
        return alt

    def status(self, stream=None) -> Tuple[int, int]:
        return pfem_get_device_status(self.cells.ws, stream, ctx=self.ctx)

    def reset_status(self, stream=None):
        pfem_reset_status(self.cells.ws, stream)

    def check(self, what: str = "device status", stream=None):
        code, detail = self.status(stream)
        if code != 0:
            raise PfemError(code, f"{what} (first failure at index {detail})")


def projection_loop(proj: Projector, pos: torch.Tensor, mesh: torch.Tensor,
                    mesh_vel: torch.Tensor, dt: float, steps: int,
                    m2p_shape=PFEM_SHAPE_LINEAR, p2m_shape=PFEM_SHAPE_QUADRATIC, solve=None,
                    incremental: bool = False, stream=None):
    """The loop of Sec. 3.1 on Zalesak's disk: each step projects the mesh field onto the
    particles (M2P), moves the particles one step with the midpoint velocity interpolated from
    mesh_vel, re-bins them (the incremental update, or a full pfem_build_cells) and projects
    the particle values back onto the mesh (P2M, shape functions rebuilt).  pos [N, 2] in
    original order; proj must have been built for pos.  Returns (pos, mesh) after `steps`."""
    for _ in range(steps):
        vals = proj.m2p(pos, mesh, shape=m2p_shape, stream=stream)
        pos = proj.advect(pos, mesh_vel, dt, stream=stream)
        if incremental:
            proj.update(pos, stream=stream)
        else:
            proj.build(pos, stream=stream)
        mesh = proj.p2m(vals, shape=p2m_shape, solve=solve, stream=stream)
    return pos, mesh


class HostRoundTrip:
    """The round trip from host memory, step after step: the positions and values of a step are
    copied from pinned host buffers, binned, projected onto the mesh (P2M) and back onto the
    particles (M2P), and the particle values are copied back into a pinned host buffer.

    The copies overlap the compute: a step's inputs go on their own stream into one of two device
    buffer sets while the previous step computes; P2M waits for the values only before its first
    kernel that reads them (the context's values event, pfem_set_values_event); the result goes
    back on a third stream while the next step runs.  step() returns at once; wait() blocks until
    the last step's result is in its host buffer.  The copies are asynchronous: a step's host
    input buffers must not be rewritten before inputs_copied() (or wait()) has returned, and
    its output buffer must not be read before wait().  proj must have a context (one is created
    if it has none)."""

    def __init__(self, proj: "Projector", C: int, dtype=torch.float32, shape=PFEM_SHAPE_QUADRATIC,
                 solve=None, m2p_shape=PFEM_SHAPE_LINEAR, stream=None):
        if proj.ctx is None:
            proj.ctx = Context()
        self.proj, self.shape, self.solve, self.m2p_shape = proj, shape, solve, m2p_shape
        dev = proj.device
        pos_t = proj.cells.pos_sorted.dtype
        self.pos_d = [torch.empty((proj.N, 2), dtype=pos_t, device=dev) for _ in range(2)]
        self.vals_d = [torch.empty((proj.N, C), dtype=dtype, device=dev) for _ in range(2)]
        self.mesh = torch.empty((proj.n, proj.n, C), dtype=dtype, device=dev)
        self.back = torch.empty((proj.N, C), dtype=dtype, device=dev)
        self.stream = stream or torch.cuda.current_stream(dev)
        self.h2d = torch.cuda.Stream(dev)
        self.d2h = torch.cuda.Stream(dev)
        ev = lambda: torch.cuda.Event()
        self.ev_pos, self.ev_vals, self.ev_free = [ev(), ev()], [ev(), ev()], [ev(), ev()]
        self.ev_done, self.ev_out = ev(), ev()
        self.k = 0

    def step(self, pos_h: torch.Tensor, vals_h: torch.Tensor, out_h: torch.Tensor):
        b = self.k & 1
        s, h2d, d2h = self.stream, self.h2d, self.d2h
        with torch.cuda.stream(h2d):
            if self.k >= 2:
                h2d.wait_event(self.ev_free[b])       # step k-2 is done with buffer set b
            self.pos_d[b].copy_(pos_h, non_blocking=True)
            self.ev_pos[b].record(h2d)
            self.vals_d[b].copy_(vals_h, non_blocking=True)
            self.ev_vals[b].record(h2d)
        s.wait_event(self.ev_pos[b])
        proj = self.proj
        proj.build(self.pos_d[b], stream=s)
        proj.ctx.set_values_event(self.ev_vals[b])
        try:
            proj.p2m(self.vals_d[b], shape=self.shape, solve=self.solve, out=self.mesh, stream=s)
        finally:
            proj.ctx.set_values_event(None)
        if self.k >= 1:
            s.wait_event(self.ev_out)                 # the previous result has left self.back
        proj.m2p(self.pos_d[b], self.mesh, out=self.back, shape=self.m2p_shape, stream=s)
        self.ev_free[b].record(s)
        self.ev_done.record(s)
        with torch.cuda.stream(d2h):
            d2h.wait_event(self.ev_done)
            out_h.copy_(self.back, non_blocking=True)
            self.ev_out.record(d2h)
        self.k += 1

    def wait(self):
        self.ev_out.synchronize()

    def inputs_copied(self):
        """Block until the last step's input copies have run (its host inputs may be reused)."""
        if self.k > 0:
            self.ev_vals[(self.k - 1) & 1].synchronize()

    def join(self, stream=None):
        """Make `stream` (default: the compute stream) wait for the last result's copy."""
        (stream or self.stream).wait_event(self.ev_out)


class Batch:
    """Device buffers and plan for many independent problems processed together.

    `sizes` is a list of (n, N) per problem; particle rows of problem p are
    [offsets[p], offsets[p+1]) of the concatenated pos/vals arrays, and its mesh is
    mesh_view(p) of the concatenated mesh output.
    """

    def __init__(self, sizes, C: int, dtype=torch.float32, device="cuda",
                 ctx: Optional[Context] = None):
        self.device = torch.device(device)
        self.ctx = ctx
        self.C, self.dtype = C, dtype
        self.problems = [(n, pfem_default_bins(n, N), N) for n, N in sizes]
        self.plan = torch.zeros((pfem_batch_plan_size(len(sizes)) + 7) // 8, dtype=torch.float64,
                                device=self.device)
        self.N_total, self.bins_total, self.nodes_total = pfem_batch_plan_init(self.problems, self.plan,
                                                                               ctx=ctx)
        dev = self.device
        self.cell_start = torch.empty(self.bins_total + 1, dtype=torch.int32, device=dev)
        self.perm = torch.empty(self.N_total, dtype=torch.int32, device=dev)
        self.pos_sorted = torch.empty((self.N_total, 2), dtype=dtype, device=dev)
        self.q_sorted = torch.empty((self.N_total, 2), dtype=torch.int32, device=dev)
        wsb = pfem_batch_workspace_size(self.N_total, self.bins_total, self.nodes_total)
        self.ws = torch.zeros((wsb + 7) // 8, dtype=torch.float64, device=dev)
        self.mesh = torch.empty((self.nodes_total, C), dtype=dtype, device=dev)
        self.back = torch.empty((self.N_total, C), dtype=dtype, device=dev)
        offs, noffs = [0], [0]
        for n, _, N in self.problems:
            offs.append(offs[-1] + N)
            noffs.append(noffs[-1] + n * n)
        self.offsets, self.node_offsets = offs, noffs
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count
        self.config = {"tile_rows": 8, "p2m_blocks": sms * 8, "m2p_blocks": sms * 16}
        self.graph = None

    def mesh_view(self, p: int) -> torch.Tensor:
        n = self.problems[p][0]
        return self.mesh[self.node_offsets[p]: self.node_offsets[p + 1]].view(n, n, self.C)

    def build(self, pos, stream=None):
        pfem_batch_build_cells(self.plan, self.N_total, self.bins_total, pos, self.cell_start,
                               self.perm, self.pos_sorted, self.q_sorted, self.ws, stream, ctx=self.ctx)

    def p2m(self, vals, shape=PFEM_SHAPE_QUADRATIC, solve=None, tile_rows=None, blocks=None,
            stream=None):
        if solve is None:
            solve = PFEM_SOLVE_F64 if vals.dtype == torch.float64 else PFEM_SOLVE_F32
        pfem_batch_project_p2m(self.plan, self.nodes_total, self.N_total, self.pos_sorted, self.q_sorted, self.cell_start,
                               self.perm, self.C, vals, shape, solve, self.mesh,
                               tile_rows or self.config["tile_rows"],
                               blocks or self.config["p2m_blocks"], self.ws, stream, ctx=self.ctx)
        return self.mesh

    def m2p(self, pos, blocks=None, stream=None):
        pfem_batch_interp_m2p(self.plan, pos, self.C, self.mesh, self.back,
                              blocks or self.config["m2p_blocks"], stream, ctx=self.ctx)
        return self.back

    def round_trip(self, pos, vals, shape=PFEM_SHAPE_QUADRATIC, solve=None, stream=None):
        self.build(pos, stream)
        self.p2m(vals, shape, solve, stream=stream)
        return self.m2p(pos, stream=stream)

    def capture(self, pos, vals, shape=PFEM_SHAPE_QUADRATIC, solve=None):
        """Capture build + P2M + M2P (tuned configuration) in a CUDA graph; replay() runs it."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.round_trip(pos, vals, shape, solve, stream=s)       # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.round_trip(pos, vals, shape, solve)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()
        return self.back

    def status(self, stream=None):
        return pfem_read_status(self.ws, stream)
