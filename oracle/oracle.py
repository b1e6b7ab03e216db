"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

The oracle restates the method of Jiang, Fang & Chen (arXiv:1204.5849) in plain C; see
map_oracle.c for the sections and equations each function follows.
"""

from __future__ import annotations

import ctypes as C
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build

SCHEMES = {"mmc": 0, "lf": 1, "weno": 2}
RIEMANN = {"lf": 0, "hllc": 1, "hlld": 2}
CONDUCTION = {"off": 0, "isotropic": 1, "aligned": 2}
LIMITERS = {"minmod": 0, "vanleer": 1, "roe": 2, "none": 3, "zero": 4}
CH_MODES = {"auto": 0, "paper": 1, "fixed": 2}
CP_MODES = {"cd": 0, "fixed": 1}
REFINE_VARS = {"rho": 1, "p": 2, "j": 4}


class orc_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("c_cfl", C.c_double), ("ch_mode", C.c_int),
                ("ch", C.c_double), ("cp_mode", C.c_int), ("c_d", C.c_double),
                ("cp", C.c_double), ("eta", C.c_double), ("eglm", C.c_int),
                ("scheme", C.c_int), ("limiter", C.c_int), ("dt_override", C.c_double),
                ("reflux", C.c_int), ("riemann", C.c_int), ("conduction", C.c_int),
                ("kappa0", C.c_double), ("subcycle", C.c_int), ("grad_t_max", C.c_double)]


class orc_problem(C.Structure):
    _fields_ = [("nbase", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3)]


class orc_refine(C.Structure):
    _fields_ = [("var_mask", C.c_int), ("thr", C.c_double), ("coarsen_thr", C.c_double),
                ("bias", C.c_double), ("filter", C.c_double), ("eps_rho", C.c_double),
                ("eps_p", C.c_double), ("eps_b", C.c_double), ("ratio", C.c_double),
                ("xi", C.c_double), ("max_level", C.c_int)]


_lib = None
_flop_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(_build.build()))
    return _lib


def flop_lib():
    """The counting build (same source, flop counters compiled in, one thread)."""
    global _flop_lib
    if _flop_lib is None:
        _flop_lib = _declare(C.CDLL(_build.build_flop_counter()))
    return _flop_lib


def _declare(L):
    if True:
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.POINTER(orc_problem), C.c_int, ip, ip]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_leaf.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_leaf.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_get_leaf_ghosted.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_fill_ghosts.argtypes = [C.c_void_p]
        L.orc_cfl.argtypes = [C.c_void_p, C.POINTER(orc_params), dp]
        L.orc_get_speeds.argtypes = [C.c_void_p, dp]
        L.orc_step.argtypes = [C.c_void_p, C.POINTER(orc_params)]
        L.orc_conduct.argtypes = [C.c_void_p, C.POINTER(orc_params), C.c_double]
        L.orc_get_dtc.argtypes = [C.c_void_p, dp]
        L.orc_flags.argtypes = [C.c_void_p, C.POINTER(orc_params), C.POINTER(orc_refine),
                                C.POINTER(C.c_byte), dp]
        L.orc_conservation.argtypes = [C.c_void_p, dp]
        L.orc_regrid.restype = C.c_void_p
        L.orc_regrid.argtypes = [C.c_void_p, C.c_int, ip, ip]
        L.orc_block_step.argtypes = [C.c_int, C.c_int, C.POINTER(orc_params), dp, C.c_double,
                                     C.c_double, C.c_double, dp, dp]
        L.orc_flux.argtypes = [C.c_int, dp, C.c_double, C.c_double, dp]
        L.orc_alpha.restype = C.c_double
        L.orc_alpha.argtypes = [C.c_int, dp, C.c_double]
        L.orc_lf_flux.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, dp]
        L.orc_hllc_flux.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, dp]
        L.orc_hlld_flux.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, dp]
        L.orc_limiter.restype = C.c_double
        L.orc_limiter.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_weno_faces.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
        L.orc_prolong_1d.restype = C.c_double
        L.orc_prolong_1d.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int]
        L.orc_flop_counts.argtypes = [C.POINTER(C.c_ulonglong), C.c_int]
    return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: Dict) -> orc_params:
    return orc_params(float(p.get("gamma", 5 / 3)), float(p.get("c_cfl", 0.4)),
                      CH_MODES[p.get("ch_mode", "auto")], float(p.get("ch", 0.0)),
                      CP_MODES[p.get("cp_mode", "cd")], float(p.get("c_d", 0.18)),
                      float(p.get("cp", 0.0)), float(p.get("eta", 0.0)), int(p.get("eglm", 1)),
                      SCHEMES[p.get("scheme", "mmc")], LIMITERS[p.get("limiter", "minmod")],
                      float(p.get("dt_override", 0.0)), int(p.get("reflux", 1)),
                      RIEMANN[p.get("riemann", "lf")], CONDUCTION[p.get("conduction", "off")],
                      float(p.get("kappa0", 0.0)), int(p.get("subcycle", 1)),
                      float(p.get("grad_t_max", 0.0)))


def make_refine(r: Dict) -> orc_refine:
    mask = 0
    for v in r.get("vars", ("rho", "p")):
        mask |= REFINE_VARS[v]
    return orc_refine(mask, float(r.get("thr", 0.2)), float(r.get("coarsen", 0.1)),
                      float(r.get("bias", 0.6)), float(r.get("filter", 0.05)),
                      float(r.get("eps_rho", 1e-12)), float(r.get("eps_p", 1e-12)),
                      float(r.get("eps_b", 0.1)), float(r.get("ratio", 2.0)),
                      float(r.get("xi", 0.0)), int(r.get("max_level", 30)))


def _problems(mesh) -> "C.Array":
    arr = (orc_problem * len(mesh.problems))()
    for q, pr in enumerate(mesh.problems):
        for d in range(3):
            arr[q].nbase[d] = int(pr.nbase[d])
            arr[q].lo[d] = float(pr.lo[d])
            arr[q].hi[d] = float(pr.hi[d])
            arr[q].bc[d][0] = int(pr.bc[d][0])
            arr[q].bc[d][1] = int(pr.bc[d][1])
    return arr


class Oracle:
    """A block mesh held by the oracle, mirroring the library's pool operations."""

    def __init__(self, mesh, state: Optional[np.ndarray] = None, _handle=None):
        self.mesh = mesh
        L = lib()
        if _handle is None:
            leaves = np.ascontiguousarray(mesh.leaves, dtype=np.int32)
            err = C.c_int(0)
            self._probs = _problems(mesh)
            h = L.orc_create(mesh.ndim, mesh.nb, len(mesh.problems), self._probs,
                             mesh.nleaves, leaves.ctypes.data_as(C.POINTER(C.c_int)), C.byref(err))
            if not h:
                raise ValueError(f"oracle rejected the mesh (code {err.value})")
            self.h = h
        else:
            self.h = _handle
        if state is not None:
            self.set_state(state)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    @property
    def block_shape(self):
        return (9,) + self.mesh.block_shape()

    def set_state(self, U: np.ndarray):
        U = np.ascontiguousarray(U, dtype=np.float64)
        for b in range(self.mesh.nleaves):
            lib().orc_set_leaf(self.h, b, _dp(U[b]))

    def get_state(self) -> np.ndarray:
        out = np.empty((self.mesh.nleaves,) + self.block_shape, dtype=np.float64)
        for b in range(self.mesh.nleaves):
            lib().orc_get_leaf(self.h, b, _dp(out[b]))
        return out

    def get_ghosted(self, leaf: int) -> np.ndarray:
        n = self.mesh.nb + 4
        nz = n if self.mesh.ndim == 3 else 1
        out = np.empty((9, nz, n, n), dtype=np.float64)
        lib().orc_get_leaf_ghosted(self.h, leaf, _dp(out))
        return out

    def fill_ghosts(self) -> int:
        return lib().orc_fill_ghosts(self.h)

    def cfl(self, params: Dict) -> np.ndarray:
        dt = np.zeros(len(self.mesh.problems))
        self._rc = lib().orc_cfl(self.h, C.byref(make_params(params)), _dp(dt))
        return dt

    def conduct(self, params: Dict, dt: float) -> int:
        """Thermal conduction alone over dt (its own time step and subcycle)."""
        return lib().orc_conduct(self.h, C.byref(make_params(params)), float(dt))

    def dtc(self) -> np.ndarray:
        out = np.zeros(len(self.mesh.problems))
        lib().orc_get_dtc(self.h, _dp(out))
        return out

    def speeds(self) -> np.ndarray:
        out = np.zeros((len(self.mesh.problems), 5))
        lib().orc_get_speeds(self.h, _dp(out))
        return out

    def step(self, params: Dict) -> int:
        return lib().orc_step(self.h, C.byref(make_params(params)))

    def advance(self, params: Dict, nsteps: int = 1) -> int:
        """fill -> cfl -> step, nsteps times (the library's step sequence)."""
        rc = 0
        for _ in range(nsteps):
            self.fill_ghosts()
            self.cfl(params)
            rc = self.step(params)
            if rc not in (0, -3):
                return rc
        return rc

    def flags(self, params: Dict, refine: Dict):
        n = self.mesh.nleaves
        f = np.zeros(n, dtype=np.int8)
        est = np.zeros(n, dtype=np.float64)
        lib().orc_flags(self.h, C.byref(make_params(params)), C.byref(make_refine(refine)),
                        f.ctypes.data_as(C.POINTER(C.c_byte)), _dp(est))
        return f, est

    def conservation(self) -> np.ndarray:
        out = np.zeros((len(self.mesh.problems), 9))
        lib().orc_conservation(self.h, _dp(out))
        return out

    def regrid(self, new_mesh) -> "Oracle":
        leaves = np.ascontiguousarray(new_mesh.leaves, dtype=np.int32)
        err = C.c_int(0)
        h = lib().orc_regrid(self.h, new_mesh.nleaves, leaves.ctypes.data_as(C.POINTER(C.c_int)),
                             C.byref(err))
        if not h:
            raise ValueError(f"oracle regrid rejected the mesh (code {err.value})")
        return Oracle(new_mesh, _handle=h)


# point-wise pieces -----------------------------------------------------------------------

def flux(d: int, w: Sequence[float], gamma: float, ch: float) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_flux(d, _dp(w), gamma, ch, _dp(f))
    return f


def alpha(d: int, w: Sequence[float], gamma: float) -> float:
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_alpha(d, _dp(w), gamma)


def lf_flux(d: int, a, b, gamma: float, ch: float) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_lf_flux(d, _dp(a), _dp(b), gamma, ch, _dp(f))
    return f


def hllc_flux(d: int, a, b, gamma: float, ch: float) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_hllc_flux(d, _dp(a), _dp(b), gamma, ch, _dp(f))
    return f


def hlld_flux(d: int, a, b, gamma: float, ch: float) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    f = np.zeros(9)
    lib().orc_hlld_flux(d, _dp(a), _dp(b), gamma, ch, _dp(f))
    return f


def limiter(kind: str, a: float, b: float) -> float:
    return lib().orc_limiter(LIMITERS[kind], a, b)


def weno_faces(um: float, u0: float, up: float):
    a = C.c_double()
    b = C.c_double()
    lib().orc_weno_faces(um, u0, up, C.byref(a), C.byref(b))
    return a.value, b.value


def prolong_1d(um: float, u0: float, up: float, odd: bool) -> float:
    return lib().orc_prolong_1d(um, u0, up, int(bool(odd)))


def block_step(ndim: int, nb: int, params: Dict, dx, dt: float, ch: float, damp: float,
               padded: np.ndarray) -> np.ndarray:
    padded = np.ascontiguousarray(padded, dtype=np.float64)
    nz = nb if ndim == 3 else 1
    out = np.empty((9, nz, nb, nb), dtype=np.float64)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    rc = lib().orc_block_step(ndim, nb, C.byref(make_params(params)), _dp(dxa), dt, ch, damp,
                              _dp(padded), _dp(out))
    if rc != 0:
        raise ValueError("oracle block step supports MMC and LF only")
    return out


# regrid decision ----------------------------------------------------------------------------

def plan_regrid(mesh, flags, max_level: int) -> np.ndarray:
    """New leaf list from per-leaf flags (+1 refine, 0 keep, -1 may coarsen), by brute force
    over sets of block keys (Sec. 4.5 refinement rule with 2:1 balance over faces, edges and
    corners).  Refine flagged leaves below max_level and, repeatedly, any leaf more than one
    level coarser than a neighbour of a new leaf; coarsen a parent whose children are all
    leaves flagged -1 and not refined, unless a block next to it ends two levels finer.
    Order: old leaf order; a refined leaf becomes its children (bits x | y<<1 | z<<2
    ascending); a coarsened parent takes the place of its first child."""
    nd = mesh.ndim
    leaves = [tuple(int(v) for v in row) for row in mesh.leaves]
    leafset = set(leaves)
    flag_of = {lf: int(f) for lf, f in zip(leaves, flags)}
    internal = set()
    for (p, L, i, j, k) in leaves:
        while L > 0:
            L -= 1
            i, j, k = i >> 1, j >> 1, k >> 1
            internal.add((p, L, i, j, k))

    def offsets():
        rz = (-1, 0, 1) if nd == 3 else (0,)
        return [(ox, oy, oz) for oz in rz for oy in (-1, 0, 1) for ox in (-1, 0, 1) if (ox, oy, oz) != (0, 0, 0)]

    def neighbour(p, L, c, off):
        q = list(c)
        for d in range(nd):
            n = mesh.problems[p].nbase[d] << L
            q[d] = c[d] + off[d]
            if q[d] < 0 or q[d] >= n:
                side = 0 if q[d] < 0 else 1
                if mesh.problems[p].bc[d][side] != 0:
                    return None
                q[d] %= n
        return tuple(q)

    def cover(p, L, q):
        """leaf covering block (L, q), or None when the region is refined below L"""
        for l in range(L, -1, -1):
            s = L - l
            key = (p, l, q[0] >> s, q[1] >> s, q[2] >> s)
            if key in leafset:
                return key
            if key in internal:
                return None
        return None

    refine = {lf for lf in leaves if flag_of[lf] > 0 and lf[1] < max_level}
    work = list(refine)
    while work:
        p, L, i, j, k = work.pop()
        for off in offsets():
            q = neighbour(p, L, (i, j, k), off)
            if q is None:
                continue
            cv = cover(p, L, q)
            if cv is not None and cv not in refine and cv[1] < L:
                refine.add(cv)
                work.append(cv)

    def children(par):
        p, L, i, j, k = par
        out = []
        for cb in range(1 << nd):
            out.append((p, L + 1, 2 * i + (cb & 1), 2 * j + ((cb >> 1) & 1),
                        2 * k + ((cb >> 2) & 1) if nd == 3 else 0))
        return out

    cand = set()
    for par in internal:
        ch = children(par)
        if all(c in leafset and flag_of[c] < 0 and c not in refine for c in ch):
            cand.add(par)
    changed = True
    while changed:
        changed = False
        for par in sorted(cand):
            p, Lp, i, j, k = par
            bad = False
            for off in offsets():
                q = neighbour(p, Lp, (i, j, k), off)
                if q is None:
                    continue
                key = (p, Lp) + q
                if key not in internal or key in cand:
                    continue
                for c in children(key):
                    # children of the neighbour that touch par
                    touch = all(not ((off[d] == 1 and ((c[2 + d] & 1) != 0)) or
                                     (off[d] == -1 and ((c[2 + d] & 1) != 1))) for d in range(nd))
                    if touch and (c in internal or c in refine):
                        bad = True
            if bad:
                cand.discard(par)
                changed = True

    out, done = [], set()
    for lf in leaves:
        p, L, i, j, k = lf
        par = (p, L - 1, i >> 1, j >> 1, k >> 1) if L > 0 else None
        if par is not None and par in cand:
            if par not in done:
                done.add(par)
                out.append(par)
        elif lf in refine:
            out.extend(children(lf))
        else:
            out.append(lf)
    return np.asarray(out, dtype=np.int32).reshape(-1, 5)


def count_step_flops(mesh, state: np.ndarray, params: Dict) -> Dict[str, float]:
    """Floating-point operations of one oracle step on ``mesh``, from the counting build.

    Returns the three raw counters and the per-cell-update figure in which every face is
    counted once: ring / ring cells + faces / (2 interior cells) + cell / interior cells.
    The update loops evaluate each face from both of its cells, so halving the face counter
    gives exactly one evaluation per face on a periodic single-level mesh.  Operations of
    the time-step reduction, the ghost fill and the state check are not counted.
    """
    L = flop_lib()
    leaves = np.ascontiguousarray(mesh.leaves, dtype=np.int32)
    err = C.c_int(0)
    probs = _problems(mesh)
    h = L.orc_create(mesh.ndim, mesh.nb, len(mesh.problems), probs, mesh.nleaves,
                     leaves.ctypes.data_as(C.POINTER(C.c_int)), C.byref(err))
    if not h:
        raise ValueError(f"oracle rejected the mesh (code {err.value})")
    cnt = (C.c_ulonglong * 3)()
    try:
        U = np.ascontiguousarray(state, dtype=np.float64)
        for q in range(mesh.nleaves):
            L.orc_set_leaf(h, q, _dp(np.ascontiguousarray(U[q])))
        L.orc_fill_ghosts(h)
        dt = np.zeros(len(mesh.problems))
        pr = make_params(params)
        L.orc_cfl(h, C.byref(pr), _dp(dt))
        if L.orc_flop_counts(cnt, 1) != 1:
            raise RuntimeError("the flop-counting oracle build has no counters")
        rc = L.orc_step(h, C.byref(pr))
        if rc != 0:
            raise RuntimeError(f"oracle step failed ({rc})")
        L.orc_flop_counts(cnt, 1)
    finally:
        L.orc_destroy(h)
    nb, nd = mesh.nb, mesh.ndim
    cells = mesh.nleaves * nb ** nd
    ring = mesh.nleaves * (nb + 2) ** nd
    ring_f, face_f, cell_f = (float(c) for c in cnt)
    return {"ring": ring_f, "face": face_f, "cell": cell_f, "cells": cells,
            "per_cell_update": ring_f / ring + face_f / (2.0 * cells) + cell_f / cells}
