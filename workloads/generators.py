"""Seeded generators: jittered particle lattices and analytic fields on the unit torus.

Conventions (shared by the CUDA path, the oracle and the tests):

* Domain: the unit periodic square [0,1)^2.
* Mesh: ``n`` x ``n`` nodes including the stored periodic image row and column,
  spacing H = 1/(n-1); node (I, J) sits at (I*H, J*H) and is stored at
  ``mesh[J, I, :]``.
* Particles: an M x M cell-centred lattice of spacing h = 1/M, each coordinate
  jittered independently by U(-a, a)*h and wrapped into [0,1).  Particle
  mu = j*M + i starts from lattice site (i, j).
* Seeds: configuration k uses SEED_BASE + k.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 1610052660
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of SplitMix64 started from ``seed``.

    SplitMix64 advances its state by the golden gamma 0x9E3779B97F4A7C15 and
    returns a bijective mix of the new state (two xor-shift-multiply rounds and a
    final xor-shift), so output i depends only on (seed, i).
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * i
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0,1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal01(seed: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform of SplitMix64 uniforms."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0,1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(2 * np.pi * u2)
    out[1::2] = r * np.sin(2 * np.pi * u2)
    return out[:count]


def jittered_lattice(M: int, a: float, seed: int) -> np.ndarray:
    """[M*M, 2] float64 positions: cell-centred M x M lattice, jitter U(-a,a)*h.

    Particle mu = j*M + i uses uniforms 2*mu (x) and 2*mu+1 (y).
    """
    N = M * M
    pos = np.empty((N, 2), dtype=np.float64)
    ii = np.tile(np.arange(M, dtype=np.float64), M)
    jj = np.repeat(np.arange(M, dtype=np.float64), M)
    if a != 0.0:
        u = uniform01(seed, 2 * N)
        xi = a * (2.0 * u[0::2] - 1.0)
        eta = a * (2.0 * u[1::2] - 1.0)
    else:
        xi = eta = 0.0
    x = (ii + 0.5 + xi) / M
    y = (jj + 0.5 + eta) / M
    pos[:, 0] = x - np.floor(x)
    pos[:, 1] = y - np.floor(y)
    return pos


def taylor_green(pos: np.ndarray, k: int = 1) -> np.ndarray:
    """[N,3] Taylor-Green vortex sheet fields (u, v, p) at wavenumber k."""
    x, y = pos[:, 0], pos[:, 1]
    w = 2.0 * np.pi * k
    out = np.empty((pos.shape[0], 3))
    out[:, 0] = np.sin(w * x) * np.cos(w * y)
    out[:, 1] = -np.cos(w * x) * np.sin(w * y)
    out[:, 2] = 0.25 * (np.cos(2 * w * x) + np.cos(2 * w * y))
    return out


def zalesak_disk(pos: np.ndarray, centre=(0.5, 0.75), radius=0.15,
                 slot_width=0.05, slot_length=0.25) -> np.ndarray:
    """[N] slotted-disk indicator: 1 inside the disk and outside the slot.

    The slot is centred on the disk's vertical axis and runs up from the bottom
    of the disk for ``slot_length``.
    """
    x, y = pos[:, 0], pos[:, 1]
    inside = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 <= radius ** 2
    slot = (np.abs(x - centre[0]) < 0.5 * slot_width) & (y < centre[1] - radius + slot_length)
    return (inside & ~slot).astype(np.float64)


def rayleigh_taylor(pos: np.ndarray, H: float) -> np.ndarray:
    """[N] density 1 below / 3 above y = 0.5 + 0.05 cos(2 pi x), tanh width 2H."""
    x, y = pos[:, 0], pos[:, 1]
    return 2.0 + np.tanh((y - 0.5 - 0.05 * np.cos(2 * np.pi * x)) / (2.0 * H))


@dataclass
class Problem:
    """One projection instance: a mesh, a particle set and particle fields."""
    name: str
    n: int                     # mesh nodes per side, image row/column included
    M: int                     # particles per side
    a: float                   # jitter amplitude in units of h
    seed: int
    pos: np.ndarray            # [N,2] float64
    vals: np.ndarray           # [N,C] float64
    channels: List[str] = field(default_factory=list)
    k: int = 1                 # Taylor-Green wavenumber
    target: Optional[np.ndarray] = None  # [n,n,C] mesh target (gradient workload)

    @property
    def N(self) -> int:
        return self.pos.shape[0]

    @property
    def C(self) -> int:
        return self.vals.shape[1]

    @property
    def H(self) -> float:
        return 1.0 / (self.n - 1)

    def nodes(self) -> np.ndarray:
        """[n,n,2] node coordinates (x = I*H, y = J*H) at mesh[J, I]."""
        g = np.arange(self.n) / (self.n - 1)
        X, Y = np.meshgrid(g, g)
        return np.stack([X, Y], axis=-1)


def _tg_problem(name, n, M, a, seed, k=1, extra_zalesak=False, channels=3):
    pos = jittered_lattice(M, a, seed)
    tg = taylor_green(pos, k)[:, :channels]
    names = ["u", "v", "p"][:channels]
    if extra_zalesak:
        tg = np.concatenate([tg, zalesak_disk(pos)[:, None]], axis=1)
        names.append("zalesak")
    return Problem(name, n, M, a, seed, pos, np.ascontiguousarray(tg), names, k)


def config_tiny() -> Problem:
    """33x33 mesh (H=1/32), 64x64 particles, jitter 0.25h, TG u,v,p in FP64."""
    return _tg_problem("tiny_33x33_64x64_tg", 33, 64, 0.25, SEED_BASE + 1)


def config_large() -> Problem:
    """1025x1025 mesh, 2048x2048 particles (h=H/2), TG u,v,p + Zalesak disk."""
    return _tg_problem("large_1025x1025_2048x2048_tg_zalesak", 1025, 2048, 0.25,
                       SEED_BASE + 2, extra_zalesak=True)


def config_precision(n: int = 4097, M: int = 8192) -> Problem:
    """4097x4097 mesh, 8192x8192 particles, Rayleigh-Taylor density step (C=1)."""
    seed = SEED_BASE + 3
    pos = jittered_lattice(M, 0.25, seed)
    rho = rayleigh_taylor(pos, 1.0 / (n - 1))[:, None]
    return Problem(f"precision_{n}x{n}_{M}x{M}_rt", n, M, 0.25, seed, pos, rho, ["rho"])


def config_batched(count: int = 256, n_lo: int = 65, n_hi: int = 513,
                   size_scale: float = 1.0) -> List[Problem]:
    """Independent uneven problems: n ~ U{n_lo..n_hi}, h/H in {1/4,1/2,1}, a=0.3,
    Taylor-Green u,v,p with k ~ U{1..8}.  ``size_scale`` < 1 shrinks n for tests."""
    seed = SEED_BASE + 4
    u = uniform01(seed, 3 * count)
    probs = []
    for p in range(count):
        n = n_lo + int(u[3 * p] * (n_hi - n_lo + 1))
        if size_scale != 1.0:
            n = max(9, int(round((n - 1) * size_scale)) + 1)
        ratio = (4, 2, 1)[int(u[3 * p + 1] * 3)]     # particles per mesh spacing
        k = 1 + int(u[3 * p + 2] * 8)
        M = (n - 1) * ratio
        probs.append(_tg_problem(f"batch{p}", n, M, 0.3, seed * 1000 + p, k=k))
    return probs


def config_grad(n: int = 1025, M: int = 2048) -> Problem:
    """Gradient workload: config-large geometry, C=1 (TG pressure), seeded target."""
    seed = SEED_BASE + 5
    pr = _tg_problem(f"grad_{n}x{n}_{M}x{M}_tgp", n, M, 0.25, seed)
    pr.vals = np.ascontiguousarray(pr.vals[:, 2:3])
    pr.channels = ["p"]
    nodes = pr.nodes().reshape(-1, 2)
    t = taylor_green(nodes)[:, 2] + 0.01 * normal01(seed + 7, nodes.shape[0])
    pr.target = t.reshape(n, n, 1)
    pr.target[-1, :, :] = pr.target[0, :, :]
    pr.target[:, -1, :] = pr.target[:, 0, :]
    return pr


def scaled_config(which: str, n: int, M: int, a: float = 0.25, seed_offset: int = 0,
                  k: int = 1) -> Problem:
    """A smaller instance of one of the workloads with the same structure."""
    if which == "tg":
        return _tg_problem(f"tg_{n}_{M}", n, M, a, SEED_BASE + 10 + seed_offset, k=k)
    if which == "tgz":
        return _tg_problem(f"tgz_{n}_{M}", n, M, a, SEED_BASE + 20 + seed_offset,
                           k=k, extra_zalesak=True)
    if which == "rt":
        seed = SEED_BASE + 30 + seed_offset
        pos = jittered_lattice(M, a, seed)
        rho = rayleigh_taylor(pos, 1.0 / (n - 1))[:, None]
        return Problem(f"rt_{n}_{M}", n, M, a, seed, pos, rho, ["rho"])
    raise ValueError(which)


def six_per_node(nc: int, a: float = 0.25, seed_offset: int = 0) -> Problem:
    """The paper's 'fine' density of six particles per mesh node (h = H/sqrt(6), Sec. 3.1,
    projFEM6 / projFEMq6): an M x M jittered lattice with M = round(sqrt(6) nc)."""
    M = int(round(np.sqrt(6.0) * nc))
    return _tg_problem(f"six_per_node_{nc + 1}_{M}", nc + 1, M, a, SEED_BASE + 40 + seed_offset)


def particles_at_nodes(nc: int, a: float = 0.0, seed: int = SEED_BASE + 50) -> Problem:
    """Particles re-created at the mesh nodes (Discussion, Eulerian-spirit variant): one
    particle per unique node, optionally jittered by U(-a, a) H per coordinate."""
    M = nc
    pos = np.empty((M * M, 2))
    ii = np.tile(np.arange(M, dtype=np.float64), M)
    jj = np.repeat(np.arange(M, dtype=np.float64), M)
    if a != 0.0:
        u = uniform01(seed, 2 * M * M)
        ii = ii + a * (2 * u[0::2] - 1)
        jj = jj + a * (2 * u[1::2] - 1)
    x, y = ii / M, jj / M
    pos[:, 0] = x - np.floor(x)
    pos[:, 1] = y - np.floor(y)
    vals = taylor_green(pos)
    return Problem(f"at_nodes_{nc + 1}", nc + 1, M, a, seed, pos, vals, ["u", "v", "p"])
