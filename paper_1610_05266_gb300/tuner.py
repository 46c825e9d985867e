"""Autotuner for the launch shapes of the batched kernels.

It times every candidate configuration on the caller's actual batch with CUDA events (after
a warm-up) and keeps the fastest; results are cached per batch signature for the process.
The candidates are the persistent P2M grid (blocks per SM), its node tile (16 x 4, 16 x 8,
16 x 16 threads) and the M2P grid.
"""
from __future__ import annotations

import itertools
from typing import Callable, Dict, Iterable, List, Tuple

import torch

_CACHE: Dict[tuple, dict] = {}


def time_ms(fn: Callable[[], None], reps: int = 3, warmup: int = 1) -> float:
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def best_of(candidates: Iterable[dict], run: Callable[[dict], None], reps: int = 3) -> Tuple[dict, List[tuple]]:
    table = []
    for cfg in candidates:
        table.append((time_ms(lambda: run(cfg), reps=reps), cfg))
    table.sort(key=lambda t: t[0])
    return table[0][1], table


def tune_batch(batch, pos, vals, shape, solve=None, reps: int = 3, quick: bool = False) -> dict:
    """Pick tile_rows / p2m_blocks / m2p_blocks for `batch` (a paper_1610_05266_gb300.Batch)."""
    key = (tuple(batch.problems), batch.C, str(vals.dtype), shape, solve)
    if key in _CACHE:
        batch.config.update({k: v for k, v in _CACHE[key].items() if not k.startswith("_")})
        return _CACHE[key]
    batch.build(pos)
    SMS = torch.cuda.get_device_properties(batch.device).multi_processor_count
    rows = (8,) if quick else (4, 8, 16)
    mult = (4, 8) if quick else (2, 4, 8, 16)
    p2m_cands = [{"tile_rows": r, "p2m_blocks": SMS * m} for r, m in itertools.product(rows, mult)]
    best_p2m, t1 = best_of(p2m_cands, lambda c: batch.p2m(vals, shape, solve, c["tile_rows"],
                                                          c["p2m_blocks"]), reps)
    m2p_cands = [{"m2p_blocks": SMS * m} for m in ((8, 16) if quick else (4, 8, 16, 32))]
    best_m2p, t2 = best_of(m2p_cands, lambda c: batch.m2p(pos, c["m2p_blocks"]), reps)
    cfg = dict(best_p2m, **best_m2p)
    cfg["_timings_ms"] = {"p2m": [(round(t, 4), c) for t, c in t1], "m2p": [(round(t, 4), c) for t, c in t2]}
    batch.config.update({k: v for k, v in cfg.items() if not k.startswith("_")})
    _CACHE[key] = cfg
    return cfg
