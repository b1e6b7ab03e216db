"""Initial conditions (closed-form functions of the cell centres) and named workloads.

Variables, in this order everywhere (Section 2, eqs. MHD-1..MHD-5):
    rho, rho*vx, rho*vy, rho*vz, Bx, By, Bz, e, psi
Three vector components are carried in 2D as well (2.5-D); psi is the GLM potential.

Only problem set-up lives here: primitives at cell centres and the definition of the
total energy density e = p/(gamma-1) + rho v^2/2 + B^2/2 (Section 2) used to turn them
into conserved variables.  Closed-form exact solutions (advected profiles, the linear
Alfven wave) are given for the tests' error measurements.
"""

from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from .mesh import (Mesh, OUTFLOW, PERIODIC, Problem, ensemble_mesh, radial_amr_mesh,
                   slab_amr_mesh, uniform_mesh)

NVAR = 9
VAR_NAMES = ("rho", "mx", "my", "mz", "bx", "by", "bz", "e", "psi")

# ---------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014), used as a counter-based generator: the value for
# a key is the output mix of (key + golden gamma).
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = np.asarray(key, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(key: np.ndarray) -> np.ndarray:
    """U[0,1) from the top 53 bits of splitmix64(key)."""
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


class _Stream:
    """Sequential draws from splitmix64 on consecutive counters of one seed."""

    def __init__(self, seed: int):
        self.base = np.uint64((seed * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF)
        self.n = 0

    def u64(self) -> int:
        with np.errstate(over="ignore"):
            v = int(splitmix64(np.array([self.base + np.uint64(self.n)], dtype=np.uint64))[0])
        self.n += 1
        return v

    def uniform(self) -> float:
        return (self.u64() >> 11) * (2.0 ** -53)


# ---------------------------------------------------------------------------------------
def conserved_from_primitive(rho, vx, vy, vz, bx, by, bz, p, gamma, psi=0.0) -> np.ndarray:
    """Stack conserved variables from primitives (e from Section 2's definition)."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    f = lambda a: np.broadcast_to(np.asarray(a, dtype=np.float64), shape)
    vx, vy, vz, bx, by, bz, p, psi = map(f, (vx, vy, vz, bx, by, bz, p, psi))
    e = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) + 0.5 * (bx * bx + by * by + bz * bz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, bx, by, bz, e, psi]).astype(np.float64)


def cell_centres(mesh: Mesh, idx: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Cell-centre coordinates of leaf ``idx`` as (z, y, x)-shaped arrays."""
    o = mesh.leaf_origin(idx)
    dx = mesh.leaf_dx(idx)
    nb = mesh.nb
    nz = nb if mesh.ndim == 3 else 1
    x = o[0] + (np.arange(nb) + 0.5) * dx[0]
    y = o[1] + (np.arange(nb) + 0.5) * dx[1]
    z = o[2] + (np.arange(nz) + 0.5) * dx[2] if mesh.ndim == 3 else np.array([0.0])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def evaluate_on_mesh(mesh: Mesh, fn: Callable, **kw) -> np.ndarray:
    """(nleaves, 9, nz, ny, nx) float64 interior data of every leaf."""
    nz, ny, nx = mesh.block_shape()
    out = np.empty((mesh.nleaves, NVAR, nz, ny, nx), dtype=np.float64)
    for b in range(mesh.nleaves):
        X, Y, Z = cell_centres(mesh, b)
        out[b] = fn(X, Y, Z, mesh=mesh, leaf=b, **kw)
    return out


# ---------------------------------------------------------------------------------------
# Initial conditions.  Each takes cell centres X, Y, Z and returns (9, ...) conserved data.

def uniform_state(X, Y, Z, gamma=5.0 / 3.0, rho=1.3, v=(0.3, -0.2, 0.1), b=(0.4, 0.25, -0.3),
                  p=0.7, psi=0.0, **_):
    one = np.ones_like(X)
    return conserved_from_primitive(rho * one, v[0], v[1], v[2], b[0], b[1], b[2], p, gamma, psi * one)


def orszag_tang(X, Y, Z, gamma=5.0 / 3.0, **_):
    """Orszag-Tang-type vortex on the periodic unit square."""
    s4 = math.sqrt(4.0 * math.pi)
    rho = np.full_like(X, 25.0 / (36.0 * math.pi))
    p = 5.0 / (12.0 * math.pi)
    vx = -np.sin(2 * math.pi * Y)
    vy = np.sin(2 * math.pi * X)
    bx = -np.sin(2 * math.pi * Y) / s4
    by = np.sin(4 * math.pi * X) / s4
    return conserved_from_primitive(rho, vx, vy, 0.0, bx, by, 0.0, p, gamma)


def alfven_wave(X, Y, Z, t=0.0, gamma=5.0 / 3.0, amp=1e-6, ndim=3, rho0=1.0, p0=0.1, **_):
    """Linear Alfven wave along the box diagonal, B0 = (1,0,0), exact at linear order.

    3D: k = 2 pi (1,1,1), e_hat = (0,1,-1)/sqrt(2).  2D: k = 2 pi (1,1), e_hat = (0,0,1).
    omega = B0.k / sqrt(rho0); dB = amp e_hat sin(k.x - omega t); dv = -dB / sqrt(rho0).
    """
    b0 = np.array([1.0, 0.0, 0.0])
    if ndim == 3:
        k = 2 * math.pi * np.array([1.0, 1.0, 1.0])
        ehat = np.array([0.0, 1.0, -1.0]) / math.sqrt(2.0)
        phase = k[0] * X + k[1] * Y + k[2] * Z
    else:
        k = 2 * math.pi * np.array([1.0, 1.0, 0.0])
        ehat = np.array([0.0, 0.0, 1.0])
        phase = k[0] * X + k[1] * Y
    omega = float(b0 @ k) / math.sqrt(rho0)
    s = amp * np.sin(phase - omega * t)
    db = [ehat[c] * s for c in range(3)]
    dv = [-db[c] / math.sqrt(rho0) for c in range(3)]
    rho = np.full_like(X, rho0)
    return conserved_from_primitive(rho, dv[0], dv[1], dv[2], b0[0] + db[0], b0[1] + db[1],
                                    b0[2] + db[2], p0, gamma)


def rotor(X, Y, Z, gamma=1.4, r0=0.1, r1=0.115, v0=2.0, **_):
    """Magnetic rotor (Section 5, 2D magnetic rotor): speed v0 at r0, linear taper to r1."""
    r = np.sqrt(X * X + Y * Y)
    f = (r1 - r) / (r1 - r0)
    inner = r < r0
    taper = (r >= r0) & (r <= r1)
    rho = np.where(inner, 10.0, np.where(taper, 1.0 + 9.0 * f, 1.0))
    rs = np.where(r > 0, r, 1.0)
    vx = np.where(inner, -v0 * Y / r0, np.where(taper, -v0 * f * Y / rs, 0.0))
    vy = np.where(inner, v0 * X / r0, np.where(taper, v0 * f * X / rs, 0.0))
    bx = 5.0 / math.sqrt(4.0 * math.pi)
    return conserved_from_primitive(rho, vx, vy, 0.0, bx, 0.0, 0.0, 1.0, gamma)


def harris_sheet(X, Y, Z, gamma=5.0 / 3.0, width=0.05, noise=1e-3, seed=1204, mesh=None, leaf=None, **_):
    """Harris current sheet with seeded velocity noise.

    The noise of a cell is 1e-3 (2U - 1) with U = uniform01 of a key built from the seed,
    the leaf level, the cell's global index at that level and the velocity component.
    """
    sech2 = 1.0 / np.cosh(Y / width) ** 2
    rho = 1.0 + sech2
    bx = np.tanh(Y / width)
    p = 0.5 * rho
    v = [np.zeros_like(X) for _ in range(3)]
    if noise and mesh is not None:
        pidx, lv, bi, bj, bk = (int(q) for q in mesh.leaves[leaf])
        prob = mesh.problems[pidx]
        nb = mesh.nb
        N = np.array(prob.nbase) * nb * 2 ** lv
        nz = nb if mesh.ndim == 3 else 1
        gk, gj, gi = np.meshgrid(bk * nb + np.arange(nz), bj * nb + np.arange(nb),
                                 bi * nb + np.arange(nb), indexing="ij")
        gidx = ((gk.astype(np.uint64) * np.uint64(N[1]) + gj.astype(np.uint64)) * np.uint64(N[0])
                + gi.astype(np.uint64))
        with np.errstate(over="ignore"):
            base = (np.uint64(seed) * np.uint64(0x100000001B3)) ^ (np.uint64(lv) << np.uint64(58))
            for c in range(3):
                key = base + gidx * np.uint64(3) + np.uint64(c)
                v[c] = noise * (2.0 * uniform01(key) - 1.0)
    return conserved_from_primitive(rho, v[0], v[1], v[2], bx, 0.0, 0.0, p, gamma)


def ensemble_modes(seed: int, nmodes: int = 8):
    """Draw (k, phase) for the rho, vx, vy and Az expansions of one ensemble problem."""
    st = _Stream(seed)
    fields = {}
    for name in ("rho", "vx", "vy", "az"):
        modes = []
        while len(modes) < nmodes:
            kx = int(st.u64() % 9) - 4
            ky = int(st.u64() % 9) - 4
            if kx == 0 and ky == 0:
                continue
            modes.append((kx, ky, 2.0 * math.pi * st.uniform()))
        fields[name] = modes
    return fields


def ensemble_problem(X, Y, Z, seed=1204, gamma=5.0 / 3.0, amp=0.1, **_):
    """Random-phase Fourier-mode state with B = curl(Az z_hat) (divergence-free)."""
    modes = ensemble_modes(seed)
    tp = 2.0 * math.pi

    def series(name):
        s = np.zeros_like(X)
        for kx, ky, ph in modes[name]:
            s += np.sin(tp * (kx * X + ky * Y) + ph) / len(modes[name])
        return s

    rho = 1.0 + amp * series("rho")
    vx = amp * series("vx")
    vy = amp * series("vy")
    bx = np.zeros_like(X)
    by = np.zeros_like(X)
    for kx, ky, ph in modes["az"]:
        kn = math.hypot(kx, ky)
        # Az = sum amp/8 cos(2 pi k.x + ph) / (2 pi |k|); Bx = dAz/dy, By = -dAz/dx
        s = np.sin(tp * (kx * X + ky * Y) + ph)
        bx += -amp / len(modes["az"]) * (ky / kn) * s
        by += amp / len(modes["az"]) * (kx / kn) * s
    return conserved_from_primitive(rho, vx, vy, 0.0, bx, by, 0.0, 1.0, gamma)


def advection_2d(X, Y, Z, t=0.0, gamma=1.4, **_):
    """Oblique density advection (Section 5, 2D accuracy test), exact at time t."""
    s3 = math.sqrt(3.0)
    xs, ys = X - t, Y - s3 * t
    rho = (np.sin(2 * math.pi * (xs + ys / s3) + math.pi / 2) + 2.0) / 3.0
    return conserved_from_primitive(rho, 1.0, s3, 0.0, 0.0, 0.0, 0.0, 1.0, gamma)


def brio_wu(X, Y, Z, gamma=2.0, **_):
    left = X < 0.0
    rho = np.where(left, 1.0, 0.125)
    by = np.where(left, 1.0, -1.0)
    p = np.where(left, 1.0, 0.1)
    return conserved_from_primitive(rho, 0.0, 0.0, 0.0, 0.75, by, 0.0, p, gamma)


def field_loop(X, Y, Z, gamma=5.0 / 3.0, b0=1e-3, r_loop=0.2, **_):
    """Field-loop advection (Section 5, 2D divergence free test)."""
    r = np.sqrt(X * X + Y * Y)
    inside = r < r_loop
    rs = np.where(r > 0, r, 1.0)
    bx = np.where(inside, -b0 * Y / rs, 0.0)
    by = np.where(inside, b0 * X / rs, 0.0)
    p = np.where(inside, 1.0 - b0 * b0 / 2.0, 1.0)
    return conserved_from_primitive(np.ones_like(X), 1.0, 1.0, 0.0, bx, by, 0.0, p, gamma)


def blast_wave(X, Y, Z, gamma=5.0 / 3.0, **_):
    """Magnetised blast wave (Section 5, 2D parallelization efficiency test)."""
    r2 = X * X + Y * Y
    p = np.where(r2 <= 0.01, 10.0, 1.0)
    b = 1.0 / math.sqrt(2.0)
    return conserved_from_primitive(np.ones_like(X), 0.0, 0.0, 0.0, b, b, 0.0, p, gamma)


def divb_bump(X, Y, Z, gamma=5.0 / 3.0, amp=1e-2, **_):
    """A non-solenoidal Bx bump in a static medium: div B != 0 initially."""
    r2 = X * X + Y * Y
    bx = amp * np.exp(-r2 / 0.01)
    return conserved_from_primitive(np.ones_like(X), 0.0, 0.0, 0.0, bx, 0.0, 0.0, 1.0, gamma)


# ---------------------------------------------------------------------------------------
# Named workloads (the benchmark configurations).  Each builder returns a dict with the
# mesh, the IC function (and its keyword arguments), method parameters and step count.

def _params(**kw):
    p = dict(gamma=5.0 / 3.0, c_cfl=0.4, scheme="mmc", limiter="minmod", eta=0.0, eglm=1,
             ch_mode="auto", ch=0.0, cp_mode="cd", c_d=0.18, cp=0.0)
    p.update(kw)
    return p


def config_ot2d(small: bool = False):
    """2D uniform 128^2 as 8x8 blocks of 16^2, MMC + minmod, Orszag-Tang, 100 steps."""
    mesh = uniform_mesh(2, 16, (8, 8))
    return dict(name="ot2d_mmc_128", mesh=mesh, ic=orszag_tang, ic_kw={},
                params=_params(scheme="mmc", limiter="minmod"), steps=100)


def config_alfven3d(small: bool = False):
    """3D uniform linear Alfven wave, 16^3 blocks, LF + van Leer, 200 steps."""
    nbb = 2 if small else 16
    mesh = uniform_mesh(3, 16, (nbb, nbb, nbb))
    return dict(name=f"alfven3d_lf_{nbb * 16}", mesh=mesh, ic=alfven_wave, ic_kw=dict(ndim=3),
                params=_params(scheme="lf", limiter="vanleer"), steps=200)


def config_rotor_amr(small: bool = False):
    """2D quadtree AMR rotor, 16^2 blocks, WENO-RK2, regrid every 4 steps (thr 0.2)."""
    if small:
        mesh = radial_amr_mesh(2, 16, (2, 2), 2, radii=(0.16, 0.34), bc=OUTFLOW)
    else:
        mesh = radial_amr_mesh(2, 16, (8, 8), 3, radii=(0.44, 0.54, 0.66), bc=OUTFLOW)
    return dict(name="rotor2d_weno_amr", mesh=mesh, ic=rotor, ic_kw={},
                params=_params(gamma=1.4, scheme="weno"), steps=100, regrid_every=4,
                refine=dict(vars=("rho", "p"), thr=0.2, coarsen=0.1, max_level=mesh.max_level))


def config_harris_amr(small: bool = False):
    """3D octree AMR Harris sheet, 8^3 blocks, resistive (eta = 1e-3), 3 levels."""
    if small:
        mesh = slab_amr_mesh(3, 8, (2, 2, 2), 1, half_widths=(0.08,))
    else:
        mesh = slab_amr_mesh(3, 8, (8, 8, 8), 2, half_widths=(0.07, 0.2))
    return dict(name="harris3d_res_amr", mesh=mesh, ic=harris_sheet, ic_kw={},
                params=_params(scheme="lf", limiter="minmod", eta=1e-3), steps=100, regrid_every=4,
                refine=dict(vars=("j",), thr=0.2, coarsen=0.1, max_level=mesh.max_level))


def ensemble_sizes(small: bool = False) -> List[int]:
    if small:
        return [32, 64, 32, 48]
    return [64] * 24 + [128] * 24 + [256] * 24 + [512] * 24


def config_ensemble(small: bool = False):
    """96 independent periodic 2D problems of uneven sizes, MMC + minmod."""
    sizes = ensemble_sizes(small)
    mesh = ensemble_mesh(16, sizes)
    return dict(name="ensemble2d_mmc_96", mesh=mesh, ic=None, ic_kw={}, ensemble_seed=1204,
                params=_params(scheme="mmc", limiter="minmod"), steps=100)


def conduction_hot_region(X, Y, Z, gamma=5.0 / 3.0, rho0=0.1, rho_hot=0.025, p0=0.1, half=0.1, **_):
    """The oblique-field conduction test's state (Sec. 5): uniform rho = 0.1, p = 0.1,
    B = (1, 1, 0), at rest, with a hot square |x|, |y| < 0.1 of rho = rho_hot (T = p/rho)."""
    hot = (np.abs(X) < half) & (np.abs(Y) < half)
    rho = np.where(hot, rho_hot, rho0)
    return conserved_from_primitive(rho, 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, p0 + 0.0 * X, gamma)


def config_conduction(small: bool = False):
    """2D field-aligned thermal conduction with subcycle, WENO + LF, 256^2 as 16x16 blocks
    of 16^2 on [-0.5, 0.5]^2, periodic, kappa0 = 1e-3 (the Sec. 5 test's parameters)."""
    n = 4 if small else 16
    mesh = uniform_mesh(2, 16, (n, n), lo=(-0.5, -0.5, 0.0), hi=(0.5, 0.5, 1.0))
    return dict(name=f"conduction2d_weno_aligned_{16 * n}", mesh=mesh, ic=conduction_hot_region, ic_kw={},
                params=_params(scheme="weno", conduction="aligned", kappa0=1e-3, subcycle=1), steps=20)


def ensemble_initial(mesh: Mesh, seed0: int = 1204) -> np.ndarray:
    """Per-problem seeded state: problem p uses seed0 + p (all blocks of a problem are
    evaluated in one call; the values do not depend on the batching)."""
    nz, ny, nx = mesh.block_shape()
    out = np.empty((mesh.nleaves, NVAR, nz, ny, nx), dtype=np.float64)
    probs = mesh.leaves[:, 0].astype(np.int64)
    for p in np.unique(probs):
        idx = np.nonzero(probs == p)[0]
        cc = [cell_centres(mesh, int(b)) for b in idx]
        X = np.stack([c[0] for c in cc])
        Y = np.stack([c[1] for c in cc])
        Z = np.stack([c[2] for c in cc])
        U = ensemble_problem(X, Y, Z, seed=seed0 + int(p))      # (9, nblocks, nz, ny, nx)
        out[idx] = np.moveaxis(U, 0, 1)
    return out


def initial_state(cfg) -> np.ndarray:
    if cfg.get("ic") is None:
        return ensemble_initial(cfg["mesh"], cfg.get("ensemble_seed", 1204))
    return evaluate_on_mesh(cfg["mesh"], cfg["ic"], **cfg.get("ic_kw", {}))


CONFIGS: Dict[str, Callable] = {
    "ot2d": config_ot2d,
    "alfven3d": config_alfven3d,
    "rotor_amr": config_rotor_amr,
    "harris_amr": config_harris_amr,
    "ensemble": config_ensemble,
    "conduction": config_conduction,
}
