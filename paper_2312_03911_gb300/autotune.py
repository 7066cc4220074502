"""Walker-tile autotuner for batches of uneven runs.

A walker tile is G lanes per walker with E components per lane (d <= G * E).
Which tile steps fastest depends on the likelihood kind and on d: more lanes
per walker shorten the per-lane work and lengthen the group reductions, more
components per lane do the opposite, and padding d up to G * E wastes lanes.
For every (kind, d) of a batch the tuner times a few iterations of that class
with each tile that pads d at most to 2 d, through the library's own walk
(ns_step), and keeps the tile with the least time per point-step.  The choice
reaches the library through its documented override GGNS_TILE_<kind>_<d>, read
when a context is created.
"""
from __future__ import annotations

import os
import time

from . import ggns

# tile id -> (G lanes per walker, E components per lane); the library's table
TILES = [(1, 2), (1, 4), (2, 4), (4, 4), (8, 4), (16, 4), (32, 4), (32, 8), (32, 16), (4, 8), (16, 2), (8, 8),
         (16, 8), (32, 1), (32, 2)]

__all__ = ["TILES", "candidates", "autotune", "apply", "env_name"]


def env_name(kind: int, d: int) -> str:
    return f"GGNS_TILE_{int(kind)}_{int(d)}"


def candidates(d: int) -> list[int]:
    """Tiles that hold d components and pad them at most to 2 d."""
    return [i for i, (g, e) in enumerate(TILES) if d <= g * e <= 2 * max(d, 2)]


def _time_class(run: dict, tile: int, warmup: int, steps: int) -> float:
    key = env_name(run["spec"]["kind"], run["spec"]["d"])
    old = os.environ.get(key)
    os.environ[key] = str(tile)
    try:
        s = ggns.Sampler([run])
        try:
            s.step(warmup)
            n0 = s.result(0, check=False)["n_like"]
            t0 = time.perf_counter()
            s.step(steps)
            n1 = s.result(0, check=False)["n_like"]  # synchronises
            dt = time.perf_counter() - t0
        finally:
            s.close()
    finally:
        if old is None:
            os.environ.pop(key, None)
        else:
            os.environ[key] = old
    return dt / max(n1 - n0, 1)


def autotune(runs: list[dict], warmup: int = 2, steps: int = 4) -> dict[tuple[int, int], int]:
    """Best tile per (kind, d) of the batch, timed on the first run of each class."""
    reps: dict[tuple[int, int], dict] = {}
    for r in runs:
        reps.setdefault((int(r["spec"]["kind"]), int(r["spec"]["d"])), r)
    choice = {}
    for (kind, d), run in reps.items():
        cands = candidates(d)
        if len(cands) == 1:
            choice[(kind, d)] = cands[0]
            continue
        cost = {t: _time_class(run, t, warmup, steps) for t in cands}
        choice[(kind, d)] = min(cost, key=cost.get)
    return choice


def apply(choice: dict[tuple[int, int], int]) -> None:
    """Make contexts created from now on use the chosen tiles."""
    for (kind, d), tile in choice.items():
        os.environ[env_name(kind, d)] = str(tile)
