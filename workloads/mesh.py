"""Block meshes: problems (domains) and their leaf blocks.

A mesh is a list of leaf blocks, each an equal-shape block of ``nb`` cells per edge
(Section 4.1: every block at every level holds the same number of cells).  A leaf is
named by (problem, level, i, j, k): at level L the problem's domain is tiled by
``nbase * 2**L`` blocks per dimension and (i, j, k) are the block's integer coordinates
in that tiling.  Several independent problems (domains) may share one mesh.

The generators below only lay out leaves; they do not implement the refinement
criterion of the method.  The refined regions are chosen geometrically (distance to a
feature) with bands wide enough that neighbouring leaves differ by at most one level.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Sequence, Tuple

import numpy as np

PERIODIC = 0
OUTFLOW = 1


@dataclass
class Problem:
    """One independent domain: base tiling, physical box and boundary kind per face."""

    nbase: Tuple[int, int, int]
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    # bc[d][s]: kind of the low (s=0) / high (s=1) face in dimension d
    bc: Tuple[Tuple[int, int], ...] = ((PERIODIC, PERIODIC),) * 3

    def dx(self, nb: int, level: int) -> np.ndarray:
        n = np.asarray(self.nbase, dtype=np.float64) * nb * (2 ** level)
        return (np.asarray(self.hi) - np.asarray(self.lo)) / n


@dataclass
class Mesh:
    ndim: int
    nb: int
    problems: List[Problem]
    leaves: np.ndarray  # (n, 5) int32: problem, level, i, j, k

    @property
    def nleaves(self) -> int:
        return int(self.leaves.shape[0])

    @property
    def cells_per_block(self) -> int:
        return self.nb ** self.ndim

    @property
    def ncells(self) -> int:
        return self.nleaves * self.cells_per_block

    @property
    def max_level(self) -> int:
        return int(self.leaves[:, 1].max()) if self.nleaves else 0

    def block_shape(self) -> Tuple[int, int, int]:
        nz = self.nb if self.ndim == 3 else 1
        return (nz, self.nb, self.nb)

    def leaf_origin(self, idx: int) -> np.ndarray:
        p, lv, i, j, k = (int(v) for v in self.leaves[idx])
        prob = self.problems[p]
        dx = prob.dx(self.nb, lv)
        return np.asarray(prob.lo) + np.array([i, j, k]) * self.nb * dx

    def leaf_dx(self, idx: int) -> np.ndarray:
        p, lv = int(self.leaves[idx, 0]), int(self.leaves[idx, 1])
        return self.problems[p].dx(self.nb, lv)


def _bc_tuple(bc, ndim):
    if isinstance(bc, int):
        return tuple((bc, bc) for _ in range(3))
    out = []
    for d in range(3):
        b = bc[d] if d < len(bc) else PERIODIC
        out.append((b, b) if isinstance(b, int) else (int(b[0]), int(b[1])))
    return tuple(out)


def uniform_mesh(ndim: int, nb: int, nbase: Sequence[int], lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0), bc=PERIODIC) -> Mesh:
    """A single-level mesh of nbase[0] x nbase[1] (x nbase[2]) blocks."""
    nbx, nby = int(nbase[0]), int(nbase[1])
    nbz = int(nbase[2]) if ndim == 3 else 1
    prob = Problem((nbx, nby, nbz), tuple(lo), tuple(hi), _bc_tuple(bc, ndim))
    leaves = [(0, 0, i, j, k) for k in range(nbz) for j in range(nby) for i in range(nbx)]
    return Mesh(ndim, nb, [prob], np.asarray(leaves, dtype=np.int32).reshape(-1, 5))


def _refine_by_target(ndim: int, nb: int, prob: Problem, pidx: int,
                      target: Callable[[np.ndarray, np.ndarray], int]) -> List[Tuple[int, ...]]:
    """Top-down split: a block at level L is split while L < target(block lo, block hi)."""
    nbz = prob.nbase[2] if ndim == 3 else 1
    lo = np.asarray(prob.lo, dtype=np.float64)
    span = np.asarray(prob.hi, dtype=np.float64) - lo
    out: List[Tuple[int, ...]] = []
    stack = [(0, i, j, k) for k in range(nbz) for j in range(prob.nbase[1])
             for i in range(prob.nbase[0])]
    stack.reverse()
    while stack:
        lv, i, j, k = stack.pop()
        nblk = np.array([prob.nbase[0], prob.nbase[1], nbz], dtype=np.float64) * 2 ** lv
        blo = lo + np.array([i, j, k]) / nblk * span
        bhi = lo + np.array([i + 1, j + 1, k + 1]) / nblk * span
        if lv < target(blo, bhi):
            kids = []
            for dk in range(2 if ndim == 3 else 1):
                for dj in range(2):
                    for di in range(2):
                        kids.append((lv + 1, 2 * i + di, 2 * j + dj, 2 * k + dk if ndim == 3 else 0))
            stack.extend(reversed(kids))
        else:
            out.append((pidx, lv, i, j, k))
    return out


def _bbox_distance_to_point(blo, bhi, ndim, c):
    d2 = 0.0
    for d in range(ndim):
        if c[d] < blo[d]:
            d2 += (blo[d] - c[d]) ** 2
        elif c[d] > bhi[d]:
            d2 += (c[d] - bhi[d]) ** 2
    return d2 ** 0.5


def radial_amr_mesh(ndim: int, nb: int, nbase: Sequence[int], max_level: int,
                    radii: Sequence[float], lo=(-0.5, -0.5, -0.5), hi=(0.5, 0.5, 0.5),
                    bc=OUTFLOW, centre=(0.0, 0.0, 0.0)) -> Mesh:
    """Refinement nested around a centre point.

    ``radii[m]`` is the distance within which blocks reach level ``max_level - m``
    (m = 0 .. max_level-1); ``radii`` must increase and consecutive radii must differ by
    at least two blocks of the coarser level so that neighbouring levels differ by one.
    """
    nbz = int(nbase[2]) if ndim == 3 else 1
    prob = Problem((int(nbase[0]), int(nbase[1]), nbz), tuple(lo), tuple(hi), _bc_tuple(bc, ndim))

    def target(blo, bhi):
        dist = _bbox_distance_to_point(blo, bhi, ndim, centre)
        for m, r in enumerate(radii):
            if dist < r:
                return max_level - m
        return 0

    leaves = _refine_by_target(ndim, nb, prob, 0, target)
    return Mesh(ndim, nb, [prob], np.asarray(leaves, dtype=np.int32).reshape(-1, 5))


def slab_amr_mesh(ndim: int, nb: int, nbase: Sequence[int], max_level: int,
                  half_widths: Sequence[float], axis: int = 1, lo=(-0.5, -0.5, -0.5),
                  hi=(0.5, 0.5, 0.5), bc=((PERIODIC, PERIODIC), (OUTFLOW, OUTFLOW),
                                          (PERIODIC, PERIODIC))) -> Mesh:
    """Refinement nested around the plane ``x[axis] = 0`` (a current sheet)."""
    nbz = int(nbase[2]) if ndim == 3 else 1
    prob = Problem((int(nbase[0]), int(nbase[1]), nbz), tuple(lo), tuple(hi), _bc_tuple(bc, ndim))

    def target(blo, bhi):
        if blo[axis] <= 0.0 <= bhi[axis]:
            dist = 0.0
        else:
            dist = min(abs(blo[axis]), abs(bhi[axis]))
        for m, w in enumerate(half_widths):
            if dist < w:
                return max_level - m
        return 0

    leaves = _refine_by_target(ndim, nb, prob, 0, target)
    return Mesh(ndim, nb, [prob], np.asarray(leaves, dtype=np.int32).reshape(-1, 5))


def ensemble_mesh(nb: int, sizes: Sequence[int], lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> Mesh:
    """Many independent periodic 2D problems of uneven sizes, one level each."""
    problems: List[Problem] = []
    leaves = []
    for p, n in enumerate(sizes):
        if n % nb:
            raise ValueError("problem size must be a multiple of the block size")
        m = n // nb
        problems.append(Problem((m, m, 1), tuple(lo), tuple(hi), _bc_tuple(PERIODIC, 2)))
        leaves.extend((p, 0, i, j, 0) for j in range(m) for i in range(m))
    return Mesh(2, nb, problems, np.asarray(leaves, dtype=np.int32).reshape(-1, 5))
