"""Shared test helpers: running the oracle to a time, error norms, mesh utilities."""

from __future__ import annotations

import math
from typing import Dict

import numpy as np


def run_to_time(o, params: Dict, T: float, max_steps: int = 100000) -> int:
    """fill -> cfl -> step until t = T (the last step shortened to land on T)."""
    t = 0.0
    n = 0
    while t < T - 1e-14 and n < max_steps:
        o.fill_ghosts()
        dt = float(o.cfl(params)[0])
        if t + dt > T:
            dt = T - t
            o.cfl(dict(params, dt_override=dt))
        o.step(params)
        t += dt
        n += 1
    return n


def l1(a: np.ndarray, b: np.ndarray) -> float:
    return float(np.abs(a - b).mean())


def per_var_rel_max(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """max |a-b| per variable divided by max |b| of that variable (1 if b == 0 there)."""
    nv = a.shape[1]
    out = np.zeros(nv)
    for v in range(nv):
        scale = float(np.abs(b[:, v]).max())
        out[v] = float(np.abs(a[:, v] - b[:, v]).max()) / (scale if scale > 0 else 1.0)
    return out


def per_var_rel_l1(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """mean |a-b| per variable divided by mean |b| of that variable (1 if b == 0 there)."""
    nv = a.shape[1]
    out = np.zeros(nv)
    for v in range(nv):
        scale = float(np.abs(b[:, v]).mean())
        out[v] = float(np.abs(a[:, v] - b[:, v]).mean()) / (scale if scale > 0 else 1.0)
    return out


def assemble_uniform(mesh, U: np.ndarray, var: int) -> np.ndarray:
    """Single-level, single-problem mesh data of one variable as a (nz, ny, nx) array."""
    nb = mesh.nb
    pr = mesh.problems[0]
    nz = pr.nbase[2] * nb if mesh.ndim == 3 else 1
    out = np.zeros((nz, pr.nbase[1] * nb, pr.nbase[0] * nb))
    bz = nb if mesh.ndim == 3 else 1
    for b, (p, lv, i, j, k) in enumerate(mesh.leaves):
        out[k * bz:(k + 1) * bz, j * nb:(j + 1) * nb, i * nb:(i + 1) * nb] = U[b, var]
    return out


def quadratic_estimate(a, b, c, h, eps, refine, X, Y):
    """The Sec. 4.5 estimator of rho = a + b x^2 + c y^2 at cell centres (X, Y), in closed
    form: the three-point first difference is 4 b x h (4 c y h) and the second difference
    2 b h^2 (2 c h^2) exactly, so |du| = sqrt(3)/2 * 4 h sqrt(b^2 x^2 + c^2 y^2) and
    |d2u| = 2 h^2 sqrt(b^2 + c^2).  Returns the first-difference part and the whole."""
    B, F = refine["bias"], refine["filter"]
    u = a + b * X * X + c * Y * Y
    du = math.sqrt(3.0) / 2.0 * 4.0 * h * np.sqrt(b * b * X * X + c * c * Y * Y)
    d2u = 2.0 * h * h * math.sqrt(b * b + c * c)
    first = B * du / (np.abs(u) + eps)
    second = (1.0 - B) * d2u / (du + F * (np.abs(u) + eps))
    return first, first + second


def two_level_mesh(n, ny_blocks, lo, hi, fine):
    """A periodic 2D mesh of n/16 x ny_blocks base blocks of 16^2 in which the blocks with
    fine(i, j, n/16) are split once (a static two-level mesh)."""
    import workloads as w
    nbx = n // 16
    prob = w.Problem((nbx, ny_blocks, 1), lo, hi)
    leaves = []
    for j in range(ny_blocks):
        for i in range(nbx):
            if fine(i, j, nbx):
                leaves += [(0, 1, 2 * i + di, 2 * j + dj, 0) for dj in range(2) for di in range(2)]
            else:
                leaves.append((0, 0, i, j, 0))
    return w.Mesh(2, 16, [prob], np.asarray(leaves, dtype=np.int32))


def advection_strip(n, refined):
    """The 1D advection strip of Table 1 (x in [-0.5, 0.5], one block high), with the middle
    half refined once when ``refined``."""
    return two_level_mesh(n, 1, (-0.5, 0, 0), (0.5, 16.0 / n, 1),
                          lambda i, j, nbx: refined and nbx // 4 <= i < 3 * nbx // 4)


def advection_1d(X, Y, Z, t=0.0, **_):
    """Table 1's density wave, (sin 2 pi (x - t) + 2) / 3 at unit speed, exact at time t."""
    from workloads.problems import conserved_from_primitive
    rho = (np.sin(2 * math.pi * (X - t)) + 2) / 3
    return conserved_from_primitive(rho, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.4)

