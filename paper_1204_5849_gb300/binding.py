"""Thin ctypes binding of the C ABI in include/map.h (argument marshalling only).

Every step of the method runs inside libmapgb300.so on the GPU.  There is no CPU
fallback: if the library is missing or no CUDA device is present, calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmapgb300.so")

MAP_OK = 0
STATUS = {0: "MAP_OK", -1: "MAP_EINVAL", -2: "MAP_ENOMEM", -3: "MAP_ECUDA", -4: "MAP_ENONFINITE",
          -5: "MAP_ENEGPRES", -6: "MAP_ETIMEOUT", -7: "MAP_EUNSUPPORTED", -8: "MAP_ESTATE"}
MAP_FP64, MAP_FP32_FIX64 = 0, 1
SCHEMES = {"mmc": 0, "lf": 1, "weno": 2}
LIMITERS = {"minmod": 0, "vanleer": 1}
RIEMANN = {"lf": 0, "hllc": 1, "hlld": 2}
CONDUCTION = {"off": 0, "isotropic": 1, "aligned": 2}
CH_MODES = {"auto": 0, "paper": 1, "fixed": 2}
CP_MODES = {"cd": 0, "fixed": 1}
REFINE_VARS = {"rho": 1, "p": 2, "j": 4}


class map_problem_desc(C.Structure):
    _fields_ = [("nbase", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("bc", (C.c_int * 2) * 3)]


class map_pool_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nb", C.c_int), ("n_ghost", C.c_int), ("precision", C.c_int),
                ("max_blocks", C.c_int), ("n_problems", C.c_int),
                ("problems", C.POINTER(map_problem_desc)), ("ext_buffer", C.c_void_p),
                ("ext_bytes", C.c_size_t)]


class map_block_desc(C.Structure):
    _fields_ = [("problem", C.c_int), ("level", C.c_int), ("ijk", C.c_int * 3)]


assert C.sizeof(map_block_desc) == 20


class map_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("c_cfl", C.c_double), ("ch_mode", C.c_int),
                ("ch", C.c_double), ("cp_mode", C.c_int), ("c_d", C.c_double), ("cp", C.c_double),
                ("eta", C.c_double), ("eglm", C.c_int), ("scheme", C.c_int), ("limiter", C.c_int),
                ("dt_override", C.c_double), ("fp64_fix_tau", C.c_double), ("reflux", C.c_int),
                ("riemann", C.c_int), ("conduction", C.c_int), ("kappa0", C.c_double),
                ("subcycle", C.c_int), ("grad_t_max", C.c_double)]


class map_tune_result(C.Structure):
    _fields_ = [("grid", C.c_int), ("w_pred", C.c_int), ("w_face", C.c_int),
                ("ms_default", C.c_double), ("ms_best", C.c_double), ("trials", C.c_int)]


class map_refine_params(C.Structure):
    _fields_ = [("var_mask", C.c_int), ("thr", C.c_double), ("coarsen_thr", C.c_double),
                ("bias", C.c_double), ("filter", C.c_double), ("eps_rho", C.c_double),
                ("eps_p", C.c_double), ("eps_b", C.c_double), ("ratio", C.c_double),
                ("xi", C.c_double), ("max_level", C.c_int)]


class MapError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "map_create_pool": (C.c_int, [C.POINTER(map_pool_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    "map_destroy_pool": (C.c_int, [C.c_void_p]),
    "map_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_set_tree": (C.c_int, [C.c_void_p, C.POINTER(map_block_desc), C.c_int]),
    "map_write_block": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "map_read_block": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "map_write_leaves": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_read_leaves": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_fill_ghosts": (C.c_int, [C.c_void_p]),
    "map_cfl_dt": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.c_void_p]),
    "map_step": (C.c_int, [C.c_void_p, C.POINTER(map_params)]),
    "map_advance": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.c_int]),
    "map_check": (C.c_int, [C.c_void_p]),
    "map_flag_refine": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.POINTER(map_refine_params),
                                  C.c_void_p, C.c_void_p]),
    "map_regrid": (C.c_int, [C.c_void_p, C.POINTER(map_block_desc), C.c_int]),
    "map_conservation": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_last_sums": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_write_leaves_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_write_leaves_async_f32": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_get_speeds_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_read_leaves_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_read_leaves_async_f32": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "map_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "map_test_fail_waits": (C.c_int, [C.c_void_p, C.c_int]),
    "map_set_conduction_loop": (C.c_int, [C.c_void_p, C.c_int]),
    "map_last_conduction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "map_get_speeds": (C.c_int, [C.c_void_p, C.c_void_p]),
    "map_kernel_launches": (C.c_longlong, [C.c_void_p]),
    "map_last_error": (C.c_char_p, [C.c_void_p]),
    "map_plan_regrid": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(map_block_desc), C.c_int,
                                  C.POINTER(C.c_int)]),
    "map_adapt": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.POINTER(map_refine_params),
                            C.POINTER(C.c_int)]),
    "map_get_leaves": (C.c_int, [C.c_void_p, C.POINTER(map_block_desc), C.c_int, C.POINTER(C.c_int)]),
    "map_cfl_dt_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                     C.POINTER(map_params), C.c_void_p, C.c_void_p]),
    "map_check_leaves": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_int, C.POINTER(map_block_desc), C.c_int,
                                   C.c_char_p, C.c_int]),
    "map_plan_leaves": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_int, C.POINTER(map_block_desc), C.c_int,
                                  C.c_void_p, C.c_int, C.POINTER(map_block_desc), C.c_int, C.POINTER(C.c_int),
                                  C.c_char_p, C.c_int]),
    "map_plan_partition": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.c_int, C.POINTER(map_block_desc), C.c_int,
                                     C.c_int, C.c_void_p, C.c_void_p, C.c_char_p, C.c_int]),
    "map_set_active": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "map_pack_leaves": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "map_unpack_leaves": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "map_local_alpha": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.c_void_p]),
    "map_set_alpha": (C.c_int, [C.c_void_p, C.POINTER(map_params), C.c_void_p]),
}

NOALLOC_MAX_BLOCKS = 65536


def cfl_dt_noalloc(u_dev_ptr: int, precision: int, ndim: int, nb: int, nblocks: int, dx,
                   params: Dict, stream: Optional[int] = None) -> np.ndarray:
    """map_cfl_dt_noalloc: (dt, c_h, c_p, damping, alpha_g) of a device-resident state."""
    L = load()
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    out = np.zeros(5, dtype=np.float64)
    rc = L.map_cfl_dt_noalloc(C.c_void_p(u_dev_ptr), precision, ndim, nb, nblocks, _ptr(dxa),
                              C.byref(make_params(params)), C.c_void_p(stream or 0), _ptr(out))
    if rc != MAP_OK:
        raise MapError(rc, "map_cfl_dt_noalloc", L.map_last_error(None).decode())
    return out


def _problems(mesh) -> "C.Array":
    probs = (map_problem_desc * len(mesh.problems))()
    for q, pr in enumerate(mesh.problems):
        for d in range(3):
            probs[q].nbase[d] = int(pr.nbase[d])
            probs[q].lo[d] = float(pr.lo[d])
            probs[q].hi[d] = float(pr.hi[d])
            probs[q].bc[d][0] = int(pr.bc[d][0])
            probs[q].bc[d][1] = int(pr.bc[d][1])
    return probs


def check_leaves(mesh) -> str:
    """map_check_leaves (host only, no GPU): '' if the leaf list is a valid tree, else why not."""
    msg = C.create_string_buffer(256)
    load().map_check_leaves(mesh.ndim, mesh.nb, _problems(mesh), len(mesh.problems), _leaves(mesh),
                            mesh.nleaves, msg, 256)
    return msg.value.decode()


def plan_leaves(mesh, flags: np.ndarray, max_level: int) -> np.ndarray:
    """map_plan_leaves (host only, no GPU): the new leaf list (n, 5) of map_plan_regrid."""
    f = np.ascontiguousarray(flags, dtype=np.int8)
    cap = int(mesh.nleaves * (8 if mesh.ndim == 3 else 4))
    arr = (map_block_desc * cap)()
    n = C.c_int(0)
    msg = C.create_string_buffer(256)
    rc = load().map_plan_leaves(mesh.ndim, mesh.nb, _problems(mesh), len(mesh.problems), _leaves(mesh),
                                mesh.nleaves, _ptr(f), int(max_level), arr, cap, C.byref(n), msg, 256)
    if rc != MAP_OK:
        raise MapError(rc, "map_plan_leaves", msg.value.decode())
    return _leaves_to_array(arr, n.value)


def plan_partition(mesh, nranks: int):
    """map_plan_partition (host only, no GPU): owner[n] (the process stepping each leaf) and
    need[nranks, n] (1 where a process needs a leaf's interior for its ghost fill)."""
    owner = np.zeros(mesh.nleaves, dtype=np.int32)
    need = np.zeros((nranks, mesh.nleaves), dtype=np.uint8)
    msg = C.create_string_buffer(256)
    rc = load().map_plan_partition(mesh.ndim, mesh.nb, _problems(mesh), len(mesh.problems), _leaves(mesh),
                                   mesh.nleaves, int(nranks), _ptr(owner), _ptr(need), msg, 256)
    if rc != MAP_OK:
        raise MapError(rc, "map_plan_partition", msg.value.decode())
    return owner, need


class Partition:
    """The leaves of a mesh cut over nranks processes (map_plan_partition) and, for one
    process, what it exchanges with each peer before its ghost fill."""

    def __init__(self, mesh, nranks: int, rank: int):
        self.nranks, self.rank = int(nranks), int(rank)
        self.owner, self.need = plan_partition(mesh, nranks)
        self.own = np.flatnonzero(self.owner == rank).astype(np.int32)

    def sends(self, peer: int) -> np.ndarray:
        """Own leaves the peer needs, in increasing caller index."""
        return np.flatnonzero((self.owner == self.rank) & (self.need[peer] != 0)).astype(np.int32)

    def recvs(self, peer: int) -> np.ndarray:
        """The peer's leaves this process needs, in increasing caller index."""
        return np.flatnonzero((self.owner == peer) & (self.need[self.rank] != 0)).astype(np.int32)

    def exchange(self, pool, dist, device) -> int:
        """Halo exchange through torch.distributed (device tensors for NCCL, CPU tensors for
        gloo): map_pack_leaves per peer, send/recv, map_unpack_leaves.  Returns the bytes
        received."""
        import torch
        dtype = torch.float64 if pool.precision == MAP_FP64 else torch.float32
        per = 9 * int(np.prod(pool.interior_shape()[1:]))
        ops, inbox = [], []
        for peer in range(self.nranks):
            if peer == self.rank:
                continue
            snd, rcv = self.sends(peer), self.recvs(peer)
            if len(snd):
                buf = torch.empty(len(snd) * per, dtype=dtype, device="cuda")
                pool.pack_leaves(snd, buf.data_ptr())
                torch.cuda.synchronize()
                ops.append(dist.P2POp(dist.isend, buf if device == "cuda" else buf.cpu(), peer))
            if len(rcv):
                buf = torch.empty(len(rcv) * per, dtype=dtype, device=device)
                ops.append(dist.P2POp(dist.irecv, buf, peer))
                inbox.append((rcv, buf))
        if ops:
            for r in dist.batch_isend_irecv(ops):
                r.wait()
        got = 0
        for rcv, buf in inbox:
            dev = buf if buf.is_cuda else buf.cuda()
            pool.unpack_leaves(rcv, dev.data_ptr())
            torch.cuda.synchronize()
            got += buf.numel() * buf.element_size()
        return got


def load(path: str = LIB_PATH):
    """Load libmapgb300.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def make_params(p: Dict) -> map_params:
    return map_params(float(p.get("gamma", 5 / 3)), float(p.get("c_cfl", 0.4)),
                      CH_MODES[p.get("ch_mode", "auto")], float(p.get("ch", 0.0)),
                      CP_MODES[p.get("cp_mode", "cd")], float(p.get("c_d", 0.18)),
                      float(p.get("cp", 0.0)), float(p.get("eta", 0.0)), int(p.get("eglm", 1)),
                      SCHEMES[p.get("scheme", "mmc")], LIMITERS[p.get("limiter", "minmod")],
                      float(p.get("dt_override", 0.0)), float(p.get("fp64_fix_tau", 1e-2)),
                      int(p.get("reflux", 1)), RIEMANN[p.get("riemann", "lf")],
                      CONDUCTION[p.get("conduction", "off")], float(p.get("kappa0", 0.0)),
                      int(p.get("subcycle", 1)), float(p.get("grad_t_max", 0.0)))


def make_refine(r: Dict) -> map_refine_params:
    mask = 0
    for v in r.get("vars", ("rho", "p")):
        mask |= REFINE_VARS[v]
    return map_refine_params(mask, float(r.get("thr", 0.2)), float(r.get("coarsen", 0.1)),
                             float(r.get("bias", 0.6)), float(r.get("filter", 0.05)),
                             float(r.get("eps_rho", 1e-12)), float(r.get("eps_p", 1e-12)),
                             float(r.get("eps_b", 0.1)), float(r.get("ratio", 2.0)),
                             float(r.get("xi", 0.0)), int(r.get("max_level", 30)))


def _leaves(mesh) -> "C.Array":
    # map_block_desc is five packed int32 (problem, level, i, j, k): one memory copy
    a = np.ascontiguousarray(np.asarray(mesh.leaves)[:, :5], dtype=np.int32)
    arr = (map_block_desc * mesh.nleaves)()
    C.memmove(arr, a.ctypes.data, a.nbytes)
    return arr


def _leaves_to_array(arr, n: int) -> np.ndarray:
    return np.frombuffer(arr, dtype=np.int32, count=5 * n).reshape(n, 5).copy()


class Pool:
    """One block pool on the current CUDA device (wraps map_create_pool .. map_destroy_pool)."""

    def __init__(self, mesh, precision: int = MAP_FP64, max_blocks: Optional[int] = None,
                 stream: Optional[int] = None, ext_buffer: Optional[int] = None, ext_bytes: int = 0):
        L = load()
        self.mesh = mesh
        self.precision = precision
        n_par_est = mesh.nleaves // (3 if mesh.ndim == 2 else 7) + 4 * len(mesh.problems) + 64
        self.max_blocks = int(max_blocks or (2 * (mesh.nleaves + n_par_est)))
        probs = _problems(mesh)
        self._probs = probs
        desc = map_pool_desc(mesh.ndim, mesh.nb, 2, precision, self.max_blocks, len(mesh.problems),
                             probs, C.c_void_p(ext_buffer or 0), ext_bytes)
        h = C.c_void_p()
        rc = L.map_create_pool(C.byref(desc), C.c_void_p(stream or 0), C.byref(h))
        if rc != MAP_OK:
            raise MapError(rc, "map_create_pool", L.map_last_error(None).decode())
        self.h = h
        self.set_tree(mesh)

    # -- plumbing
    def _ck(self, rc: int, what: str):
        if rc != MAP_OK:
            raise MapError(rc, what, load().map_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            load().map_destroy_pool(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nleaves(self) -> int:
        return self.mesh.nleaves

    def interior_shape(self):
        return (9,) + self.mesh.block_shape()

    # -- ABI calls
    def set_stream(self, stream: Optional[int]):
        self._ck(load().map_set_stream(self.h, C.c_void_p(stream or 0)), "map_set_stream")

    def set_tree(self, mesh):
        self._leaves_arr = _leaves(mesh)
        self._ck(load().map_set_tree(self.h, self._leaves_arr, mesh.nleaves), "map_set_tree")
        self.mesh = mesh

    def write_block(self, leaf: int, u: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        self._ck(load().map_write_block(self.h, leaf, _ptr(u)), "map_write_block")

    def read_block(self, leaf: int) -> np.ndarray:
        out = np.empty(self.interior_shape(), dtype=np.float64)
        self._ck(load().map_read_block(self.h, leaf, _ptr(out)), "map_read_block")
        return out

    def write_leaves(self, U: np.ndarray):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == (self.nleaves,) + self.interior_shape()
        self._ck(load().map_write_leaves(self.h, _ptr(U)), "map_write_leaves")

    def write_leaves_ptr(self, host_ptr: int):
        self._ck(load().map_write_leaves(self.h, C.c_void_p(host_ptr)), "map_write_leaves")

    def write_leaves_async_ptr(self, host_ptr: int):
        """Asynchronous write from host memory (see map_write_leaves_async)."""
        self._ck(load().map_write_leaves_async(self.h, C.c_void_p(host_ptr)), "map_write_leaves_async")

    def write_leaves_async_f32_ptr(self, host_ptr: int):
        """Asynchronous write from an FP32 host layout (see map_write_leaves_async_f32)."""
        self._ck(load().map_write_leaves_async_f32(self.h, C.c_void_p(host_ptr)), "map_write_leaves_async_f32")

    def read_leaves_async_ptr(self, host_ptr: int):
        """Asynchronous read of the state into host memory (see map_read_leaves_async)."""
        self._ck(load().map_read_leaves_async(self.h, C.c_void_p(host_ptr)), "map_read_leaves_async")

    def read_leaves_async_f32_ptr(self, host_ptr: int):
        """Asynchronous read into an FP32 host layout (see map_read_leaves_async_f32)."""
        self._ck(load().map_read_leaves_async_f32(self.h, C.c_void_p(host_ptr)), "map_read_leaves_async_f32")

    def speeds_async_ptr(self, host_ptr: int):
        """Asynchronous read of [n_problems][5] speeds into host memory at host_ptr."""
        self._ck(load().map_get_speeds_async(self.h, C.c_void_p(host_ptr)), "map_get_speeds_async")

    def read_leaves(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty((self.nleaves,) + self.interior_shape(), dtype=np.float64)
        self._ck(load().map_read_leaves(self.h, _ptr(out)), "map_read_leaves")
        return out

    def read_leaves_ptr(self, host_ptr: int):
        self._ck(load().map_read_leaves(self.h, C.c_void_p(host_ptr)), "map_read_leaves")

    def fill_ghosts(self):
        self._ck(load().map_fill_ghosts(self.h), "map_fill_ghosts")

    def cfl_dt(self, params: Dict) -> np.ndarray:
        dt = np.zeros(len(self.mesh.problems))
        self._ck(load().map_cfl_dt(self.h, C.byref(make_params(params)), _ptr(dt)), "map_cfl_dt")
        return dt

    def step(self, params: Dict):
        self._ck(load().map_step(self.h, C.byref(make_params(params))), "map_step")

    def advance(self, params: Dict, nsteps: int = 1):
        self._ck(load().map_advance(self.h, C.byref(make_params(params)), int(nsteps)), "map_advance")

    def check(self) -> int:
        return load().map_check(self.h)

    def flag_refine(self, params: Dict, refine: Dict):
        f = np.zeros(self.nleaves, dtype=np.int8)
        est = np.zeros(self.nleaves, dtype=np.float64)
        self._ck(load().map_flag_refine(self.h, C.byref(make_params(params)), C.byref(make_refine(refine)),
                                        _ptr(f), _ptr(est)), "map_flag_refine")
        return f, est

    def regrid(self, new_mesh):
        arr = _leaves(new_mesh)
        self._ck(load().map_regrid(self.h, arr, new_mesh.nleaves), "map_regrid")
        self._leaves_arr = arr
        self.mesh = new_mesh

    def plan_regrid(self, flags: np.ndarray, max_level: int) -> np.ndarray:
        """The new leaf list (n, 5) decided from per-leaf flags (map_plan_regrid)."""
        f = np.ascontiguousarray(flags, dtype=np.int8)
        cap = int(self.nleaves * (8 if self.mesh.ndim == 3 else 4))
        arr = (map_block_desc * cap)()
        n = C.c_int(0)
        self._ck(load().map_plan_regrid(self.h, _ptr(f), int(max_level), arr, cap, C.byref(n)), "map_plan_regrid")
        return _leaves_to_array(arr, n.value)

    def get_leaves(self) -> np.ndarray:
        cap = self.nleaves
        arr = (map_block_desc * cap)()
        n = C.c_int(0)
        self._ck(load().map_get_leaves(self.h, arr, cap, C.byref(n)), "map_get_leaves")
        return _leaves_to_array(arr, n.value)

    def adapt(self, params: Dict, refine: Dict):
        """flags -> plan -> regrid (map_adapt); the pool's mesh follows the new leaves."""
        n = C.c_int(0)
        self._ck(load().map_adapt(self.h, C.byref(make_params(params)), C.byref(make_refine(refine)),
                                  C.byref(n)), "map_adapt")
        cap = n.value
        arr = (map_block_desc * cap)()
        m = C.c_int(0)
        self._ck(load().map_get_leaves(self.h, arr, cap, C.byref(m)), "map_get_leaves")
        from dataclasses import replace
        self.mesh = replace(self.mesh, leaves=_leaves_to_array(arr, m.value))
        self._leaves_arr = arr
        return self.mesh

    def conservation(self) -> np.ndarray:
        out = np.zeros((len(self.mesh.problems), 9))
        self._ck(load().map_conservation(self.h, _ptr(out)), "map_conservation")
        return out

    def last_conduction(self):
        """(dt_c per problem, conduction substeps of the last step per problem)."""
        dtc = np.zeros(len(self.mesh.problems))
        n = np.zeros(len(self.mesh.problems), dtype=np.int32)
        self._ck(load().map_last_conduction(self.h, _ptr(dtc), n.ctypes.data_as(C.c_void_p)),
                 "map_last_conduction")
        return dtc, n

    def last_sums(self) -> np.ndarray:
        """Conservation sums reduced by the last map_advance step (no extra pass)."""
        out = np.zeros((len(self.mesh.problems), 9))
        self._ck(load().map_last_sums(self.h, _ptr(out)), "map_last_sums")
        return out

    def autotune(self, params: Dict, reps: int = 3) -> Dict:
        """Pick the step kernel's launch shape for this pool (see map_autotune)."""
        r = map_tune_result()
        self._ck(load().map_autotune(self.h, C.byref(make_params(params)), int(reps), C.byref(r)),
                 "map_autotune")
        return {"grid": r.grid, "w_pred": r.w_pred, "w_face": r.w_face, "ms_default": r.ms_default,
                "ms_best": r.ms_best, "trials": r.trials}

    def test_fail_waits(self, on):
        """Test hook (map_test_fail_waits): True / 1 every bounded wait gives up at once, 2 only
        the conduction loop's grid barrier, False / 0 normal waits."""
        self._ck(load().map_test_fail_waits(self.h, 2 if on == 2 else (1 if on else 0)), "map_test_fail_waits")

    def set_conduction_loop(self, on: bool):
        """Conduction substeps in one cooperative launch where the pool allows it (default),
        or one fill and one kernel per substep (map_set_conduction_loop)."""
        self._ck(load().map_set_conduction_loop(self.h, 1 if on else 0), "map_set_conduction_loop")

    def set_launch(self, grid: int = 0, w_pred: int = 0, w_face: int = 0):
        self._ck(load().map_set_launch(self.h, int(grid), int(w_pred), int(w_face)), "map_set_launch")

    # -- partitioned pools (map_set_active and the calls around it)
    def set_active(self, leaves):
        if leaves is None:
            self._ck(load().map_set_active(self.h, None, -1), "map_set_active")
            return
        a = np.ascontiguousarray(leaves, dtype=np.int32)
        self._ck(load().map_set_active(self.h, _ptr(a), len(a)), "map_set_active")

    def pack_leaves(self, leaves, dev_ptr: int):
        a = np.ascontiguousarray(leaves, dtype=np.int32)
        self._ck(load().map_pack_leaves(self.h, _ptr(a), len(a), C.c_void_p(dev_ptr)), "map_pack_leaves")

    def unpack_leaves(self, leaves, dev_ptr: int):
        a = np.ascontiguousarray(leaves, dtype=np.int32)
        self._ck(load().map_unpack_leaves(self.h, _ptr(a), len(a), C.c_void_p(dev_ptr)), "map_unpack_leaves")

    def local_alpha(self, params: Dict) -> np.ndarray:
        out = np.zeros(len(self.mesh.problems))
        self._ck(load().map_local_alpha(self.h, C.byref(make_params(params)), _ptr(out)), "map_local_alpha")
        return out

    def set_alpha(self, params: Dict, alpha):
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        self._ck(load().map_set_alpha(self.h, C.byref(make_params(params)), _ptr(a)), "map_set_alpha")

    def speeds(self) -> np.ndarray:
        out = np.zeros((len(self.mesh.problems), 5))
        self._ck(load().map_get_speeds(self.h, _ptr(out)), "map_get_speeds")
        return out

    def kernel_launches(self) -> int:
        return int(load().map_kernel_launches(self.h))
