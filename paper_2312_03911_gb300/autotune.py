"""Walker-tile autotuner for batches of uneven runs.

A walker tile is G lanes per walker with E components per lane (d <= G * E), so
32 / G walkers share a warp.  Which tile steps fastest depends on the likelihood
kind and on d: more lanes per walker shorten the per-lane work and lengthen the
group reductions, more components per lane do the opposite, and padding d up to
G * E wastes lanes.  Dense likelihoods whose precision matrix exceeds shared
memory have a second choice: one walker per warp with a CTA of walkers sharing
each tile of P (cooperative), or every walker reading P on its own.  For every
(kind, d) of a batch the tuner times a few iterations of that class with each
tile that pads d at most to 2 d (and, for those dense classes, both layouts)
through the library's own walk (ns_step), and keeps the choice with the least
time per point-step.  The choice reaches the library through the run's
configuration (ns_config.tile and ns_config.coop).
"""
from __future__ import annotations

import time

from . import ggns

# tile id -> (G lanes per walker, E components per lane); the library's table
TILES = [(1, 2), (1, 4), (2, 4), (4, 4), (8, 4), (16, 4), (32, 4), (32, 8), (32, 16), (4, 8), (16, 2), (8, 8),
         (16, 8), (32, 1), (32, 2)]

__all__ = ["TILES", "candidates", "autotune", "apply"]


def candidates(d: int) -> list[int]:
    """Tiles that hold d components and pad them at most to 2 d."""
    return [i for i, (g, e) in enumerate(TILES) if d <= g * e <= 2 * max(d, 2)]


def _layouts(run: dict) -> list[int]:
    """coop values worth timing: both layouts for dense kinds at d > 128, else the default."""
    dense = int(run["spec"]["kind"]) in (ggns.LIK_DENSE_GAUSS, ggns.LIK_DENSE_MIX)
    return [0, -1] if dense and int(run["spec"]["d"]) > 128 else [0]


def _time_class(run: dict, tile: int, coop: int, warmup: int, steps: int) -> float:
    r = dict(run, cfg=dict(run.get("cfg", {}), tile=tile + 1, coop=coop))
    s = ggns.Sampler([r])
    try:
        s.step(warmup)
        n0 = s.result(0, check=False)["n_like"]
        t0 = time.perf_counter()
        s.step(steps)
        n1 = s.result(0, check=False)["n_like"]  # synchronises
        dt = time.perf_counter() - t0
    finally:
        s.close()
    return dt / max(n1 - n0, 1)


def autotune(runs: list[dict], warmup: int = 2, steps: int = 4) -> dict[tuple[int, int], tuple[int, int]]:
    """Best (tile, coop) per (kind, d) of the batch, timed on the first run of each class."""
    reps: dict[tuple[int, int], dict] = {}
    for r in runs:
        reps.setdefault((int(r["spec"]["kind"]), int(r["spec"]["d"])), r)
    choice = {}
    for (kind, d), run in reps.items():
        opts = [(t, c) for t in candidates(d) for c in _layouts(run)]
        if len(opts) == 1:
            choice[(kind, d)] = opts[0]
            continue
        cost = {o: _time_class(run, o[0], o[1], warmup, steps) for o in opts}
        choice[(kind, d)] = min(cost, key=cost.get)
    return choice


def apply(choice: dict[tuple[int, int], tuple[int, int]], runs: list[dict]) -> list[dict]:
    """The runs with the chosen tile (ns_config.tile = id + 1) and layout in their configuration."""
    out = []
    for r in runs:
        key = (int(r["spec"]["kind"]), int(r["spec"]["d"]))
        if key in choice:
            tile, coop = choice[key]
            r = dict(r, cfg=dict(r.get("cfg", {}), tile=tile + 1, coop=coop))
        out.append(r)
    return out
