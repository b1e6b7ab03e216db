"""Block-tile shape choice for a uniform domain, on top of the launch-shape autotuner.

map_autotune (the C ABI) picks the step kernel's grid and warp schedule for a given pool.
The block edge itself (8 or 16 cells per block) is fixed when the mesh is built, so it is
chosen here: the same domain is built with each candidate block edge, the launch shape of
each pool is tuned, and a few batched steps are timed on the device.
"""

from __future__ import annotations

import time
from typing import Callable, Dict, Sequence, Tuple

from .binding import MAP_FP32_FIX64, Pool


def choose_block_size(make_mesh: Callable[[int], object], make_state: Callable[[object], object],
                      params: Dict, precision: int = MAP_FP32_FIX64, candidates: Sequence[int] = (8, 16),
                      steps: int = 5, reps: int = 2) -> Tuple[int, Dict[int, Dict]]:
    """Returns (best block edge, per candidate {ms_per_step, launch shape}).

    make_mesh(nb) builds the domain with blocks of nb cells per edge (the same cells for
    every candidate); make_state(mesh) its initial state (n_leaves, 9, nz, nb, nb).
    """
    report: Dict[int, Dict] = {}
    for nb in candidates:
        mesh = make_mesh(nb)
        pool = Pool(mesh, precision, max_blocks=mesh.nleaves)
        try:
            pool.write_leaves(make_state(mesh))
            shape = pool.autotune(params, reps=reps)
            pool.advance(params, 1)                      # capture the step graph
            pool.check()
            t0 = time.perf_counter()
            pool.advance(params, steps)
            pool.check()                                 # synchronises
            ms = 1e3 * (time.perf_counter() - t0) / steps
            report[nb] = {"ms_per_step": ms, "cells": mesh.ncells, **shape}
        finally:
            pool.close()
    best = min(report, key=lambda k: report[k]["ms_per_step"] / report[k]["cells"])
    return best, report
