"""ctypes front end of ``pfem_oracle.c`` (plain FP64 CPU oracle; test infrastructure only).

Every function mirrors one C entry point; see the C file for what each computes and the
paper passage it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pfem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
KSTEN = 96  # stencil capacity per edge (OR_KSTEN)

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_ip = ctypes.POINTER(ctypes.c_int)

_STATUS = {0: "OK", 1: "invalid argument", 4: "capacity (window) exceeded", 5: "degenerate input"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {_STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP) into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        i64, i32 = ctypes.c_int64, ctypes.c_int
        L.or_build_cells.argtypes = [i32, i64, _f64p, _i32p, _i32p, _u32p]
        L.or_node_weights.argtypes = [i32, i64, _f64p, _i32p, _i32p, _u32p, i32, i32, i32, i32,
                                      _i32p, _f64p, _ip, _i32p, _ip]
        L.or_node_edges.argtypes = [i32, i64, _f64p, _i32p, _i32p, _u32p, i32, i32, _i32p, _f64p,
                                    _i32p, _f64p, _ip, _ip]
        L.or_node_weight_derivs.argtypes = [i32, i64, _f64p, _i32p, _i32p, _u32p, i32, i32, i32,
                                            i64, i32, i32, _i32p, _f64p, _ip]
        L.or_star.argtypes = [i32, i64, _f64p, _i32p, _i32p, _u32p, i64, _i32p, i32, _ip]
        L.or_p2m.argtypes = [i32, i64, _f64p, i32, _f64p, i32, _f64p, i32, i64, i64]
        L.or_m2p.argtypes = [i32, i64, _f64p, i32, _f64p, _f64p]
        L.or_p2m_backward.argtypes = [i32, i64, _f64p, i32, _f64p, i32, _f64p, _f64p, _f64p,
                                      i64, i64]
        L.or_m2p_backward.argtypes = [i32, i64, _f64p, i32, _f64p, _f64p, _f64p, _f64p]
        L.or_m2p_quadratic.argtypes = [i32, i64, _f64p, i32, _f64p, _f64p]
        L.or_mesh_edge.argtypes = [i32, _i32p, _f64p]
        _lib = L
    return _lib


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(code, what)


def _pos(pos) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 2))


def fixed_point(x) -> np.ndarray:
    """round(x * 2^32) mod 2^32 (round half to even), as uint32."""
    v = np.rint(np.ldexp(np.asarray(x, dtype=np.float64), 32)).astype(np.int64)
    return (v & 0xFFFFFFFF).astype(np.uint32)


class Cells:
    """The oracle's cell list: cell_start [(n-1)^2+1], perm [N], qs [N,2] uint32."""

    def __init__(self, n: int, pos: np.ndarray):
        pos = _pos(pos)
        self.n, self.N, self.pos = n, pos.shape[0], pos
        self.cell_start = np.zeros((n - 1) * (n - 1) + 1, np.int32)
        self.perm = np.zeros(max(self.N, 1), np.int32)
        self.qs = np.zeros((max(self.N, 1), 2), np.uint32)
        _check(lib().or_build_cells(n, self.N, pos, self.cell_start, self.perm, self.qs),
               "build_cells")
        self.perm = self.perm[: self.N]
        self.qs = self.qs[: self.N]

    def args(self):
        return (self.n, self.N, self.pos, self.cell_start, np.ascontiguousarray(self.perm),
                np.ascontiguousarray(self.qs))


def build_cells(n: int, pos) -> Cells:
    return Cells(n, pos)


def node_weights(cells: Cells, I: int, J: int, shape: int = 1, kmax: int = 128):
    """(idx [k] original particle indices, w [k], tri [3], min_rank) of node (I, J)."""
    idx = np.zeros(kmax, np.int32)
    w = np.zeros(kmax)
    tri = np.zeros(3, np.int32)
    cnt, rank = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().or_node_weights(*cells.args(), I, J, shape, kmax, idx, w, ctypes.byref(cnt),
                                 tri, ctypes.byref(rank)), "node_weights")
    k = cnt.value
    return idx[:k].copy(), w[:k].copy(), tri.copy(), rank.value


def node_edges(cells: Cells, I: int, J: int):
    """Per-edge detail: tri [3], lam [3], list of (stencil idx, A) for edges (e, e+1), ranks."""
    tri = np.zeros(3, np.int32)
    lam = np.zeros(3)
    st = np.zeros(3 * KSTEN, np.int32)
    A = np.zeros(3 * KSTEN)
    k = (ctypes.c_int * 3)()
    rank = (ctypes.c_int * 3)()
    _check(lib().or_node_edges(*cells.args(), I, J, tri, lam, st, A,
                               ctypes.cast(k, _ip), ctypes.cast(rank, _ip)), "node_edges")
    edges = [(st[e * KSTEN: e * KSTEN + k[e]].copy(), A[e * KSTEN: e * KSTEN + k[e]].copy())
             for e in range(3)]
    return tri, lam, edges, [rank[e] for e in range(3)]


def node_weight_derivs(cells: Cells, I: int, J: int, m: int, dim: int, shape: int = 1,
                       kmax: int = 128):
    """Complex-step d w_{(I,J) mu} / d pos[m, dim] for the node's weight set."""
    idx = np.zeros(kmax, np.int32)
    dw = np.zeros(kmax)
    cnt = ctypes.c_int(0)
    _check(lib().or_node_weight_derivs(*cells.args(), I, J, shape, m, dim, kmax, idx, dw,
                                       ctypes.byref(cnt)), "node_weight_derivs")
    return idx[: cnt.value].copy(), dw[: cnt.value].copy()


def star(cells: Cells, m: int, kmax: int = 32) -> np.ndarray:
    """Counter-clockwise Delaunay neighbours (original indices) of original particle m."""
    out = np.zeros(kmax, np.int32)
    cnt = ctypes.c_int(0)
    _check(lib().or_star(*cells.args(), m, out, kmax, ctypes.byref(cnt)), "star")
    return out[: cnt.value].copy()


def p2m(n: int, pos, vals, shape: int = 1, nthreads: int = 1,
        node_range: Optional[Tuple[int, int]] = None) -> np.ndarray:
    """Eq. (p2m) at all n x n nodes -> [n, n, C] (nodes outside node_range left at 0)."""
    pos = _pos(pos)
    vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64).reshape(pos.shape[0], -1))
    C = vals.shape[1]
    mesh = np.zeros((n * n, C))
    b, e = node_range if node_range is not None else (0, -1)
    _check(lib().or_p2m(n, pos.shape[0], pos, C, vals, shape, mesh, nthreads, b, e), "p2m")
    return mesh.reshape(n, n, C)


def mesh_edge(edge_type: int):
    """(node offsets [k,2] from the edge's first node, coefficients A [k]) of a mesh edge of
    direction (1,0), (0,1) or (1,1) (edge_type 0, 1, 2)."""
    off = np.zeros(32, np.int32)
    A = np.zeros(16)
    k = lib().or_mesh_edge(edge_type, off, A)
    if k < 0:
        raise OracleError(1, "mesh_edge")
    return off[: 2 * k].reshape(k, 2).copy(), A[:k].copy()


def m2p_quadratic(n: int, pos, mesh) -> np.ndarray:
    """M2P with quadratically consistent mesh shape functions -> [N, C]."""
    pos = _pos(pos)
    mesh = np.ascontiguousarray(np.asarray(mesh, dtype=np.float64).reshape(n * n, -1))
    C = mesh.shape[1]
    vals = np.zeros((pos.shape[0], C))
    _check(lib().or_m2p_quadratic(n, pos.shape[0], pos, C, mesh, vals), "m2p_quadratic")
    return vals


def m2p(n: int, pos, mesh) -> np.ndarray:
    """Eq. (m2p) with linear FE on the structured mesh -> [N, C]."""
    pos = _pos(pos)
    mesh = np.ascontiguousarray(np.asarray(mesh, dtype=np.float64).reshape(n * n, -1))
    C = mesh.shape[1]
    vals = np.zeros((pos.shape[0], C))
    _check(lib().or_m2p(n, pos.shape[0], pos, C, mesh, vals), "m2p")
    return vals


def p2m_backward(n: int, pos, vals, grad_mesh, shape: int = 1,
                 node_range: Optional[Tuple[int, int]] = None):
    """(grad_vals [N,C], grad_pos [N,2]) of P2M for upstream gradient grad_mesh [n,n,C]."""
    pos = _pos(pos)
    N = pos.shape[0]
    vals = np.ascontiguousarray(np.asarray(vals, dtype=np.float64).reshape(N, -1))
    C = vals.shape[1]
    gm = np.ascontiguousarray(np.asarray(grad_mesh, dtype=np.float64).reshape(n * n, C))
    gv = np.zeros((N, C))
    gp = np.zeros((N, 2))
    b, e = node_range if node_range is not None else (0, -1)
    _check(lib().or_p2m_backward(n, N, pos, C, vals, shape, gm, gv, gp, b, e), "p2m_backward")
    return gv, gp


def m2p_backward(n: int, pos, mesh, grad_vals):
    """(grad_mesh [n,n,C], grad_pos [N,2]) of M2P for upstream gradient grad_vals [N,C]."""
    pos = _pos(pos)
    N = pos.shape[0]
    mesh = np.ascontiguousarray(np.asarray(mesh, dtype=np.float64).reshape(n * n, -1))
    C = mesh.shape[1]
    gv = np.ascontiguousarray(np.asarray(grad_vals, dtype=np.float64).reshape(N, C))
    gm = np.zeros((n * n, C))
    gp = np.zeros((N, 2))
    _check(lib().or_m2p_backward(n, N, pos, C, mesh, gv, gm, gp), "m2p_backward")
    return gm.reshape(n, n, C), gp


def advect_midpoint(n: int, pos, mesh_vel, dt: float) -> np.ndarray:
    """One midpoint step (the scheme of Sec. 3.2; the move of the Sec. 3.1 loop on Zalesak's
    disk) of particles in the velocity field mesh_vel [n, n, 2], interpolated by eq. (m2p) with
    linear FE: r_half = r + dt/2 u(r), r_new = r + dt u(r_half), wrapped into [0, 1)."""
    pos = _pos(pos)
    u = m2p(n, pos, mesh_vel)
    half = pos + 0.5 * dt * u
    new = pos + dt * m2p(n, half, mesh_vel)
    return new - np.floor(new)
