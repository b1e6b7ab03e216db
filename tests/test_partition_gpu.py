"""The partitioned step on the GPU (Sec. 4.2 load balance, Sec. 4.3 boundary conditions
between processes), with the processes emulated as pools in one process on one GPU.

Each emulated process has a pool holding only its own leaves (the rest NaN), steps only
them (map_set_active), receives its halo leaves from its peers' pools through device
buffers (map_pack_leaves / map_unpack_leaves: the transfer a process would make with NCCL),
and takes the maximum of the peers' signal speeds (map_local_alpha, map_set_alpha: the
all-reduce).  After several steps its own leaves must equal, bitwise, those of one pool
stepping everything, and its dt the single pool's.  No kernel of one pool waits for another:
the host orders every transfer.  A second test runs two real processes on the one GPU,
exchanging through gloo (host copies), with the library's Partition.exchange.
"""

from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import workloads as w
from workloads.problems import ensemble_problem, harris_sheet, rotor

pytestmark = pytest.mark.gpu

CASES = {
    "3d_periodic_16": (lambda: w.uniform_mesh(3, 16, (2, 2, 2)),
                       lambda m: w.evaluate_on_mesh(m, w.alfven_wave, ndim=3, amp=1e-2)),
    "2d_periodic_16": (lambda: w.uniform_mesh(2, 16, (4, 3)),
                       lambda m: w.evaluate_on_mesh(m, lambda X, Y, Z, **_: ensemble_problem(X, Y, Z, seed=3))),
    "2d_amr_outflow_8": (lambda: w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.OUTFLOW),
                         lambda m: w.evaluate_on_mesh(m, rotor)),
    "3d_amr_slab_8": (lambda: w.slab_amr_mesh(3, 8, (2, 2, 2), 1, half_widths=(0.08,)),
                      lambda m: w.evaluate_on_mesh(m, harris_sheet)),
}


def _params(name, scheme):
    p = dict(gamma=5 / 3, c_cfl=0.4, scheme=scheme, limiter="vanleer" if scheme == "lf" else "minmod",
             eglm=1, eta=1e-3 if name.startswith("3d_amr") else 0.0, reflux=0)
    if name == "2d_amr_outflow_8":
        p["gamma"] = 1.4
    return p


def _exchange(pools, parts, prec):
    """Every pool sends each peer the own leaves the peer needs (pack -> device buffer ->
    unpack), in rank order."""
    import torch
    dtype = torch.float64 if prec == 0 else torch.float32
    per = 9 * int(np.prod(pools[0].interior_shape()[1:]))
    moved = 0
    for r, (pool, part) in enumerate(zip(pools, parts)):
        for q in range(len(pools)):
            if q == r:
                continue
            snd = part.sends(q)
            if not len(snd):
                continue
            buf = torch.empty(len(snd) * per, dtype=dtype, device="cuda:0")
            pool.pack_leaves(snd, buf.data_ptr())
            torch.cuda.synchronize()
            np.testing.assert_array_equal(parts[q].recvs(r), snd)
            pools[q].unpack_leaves(snd, buf.data_ptr())
            torch.cuda.synchronize()
            moved += len(snd)
    return moved


@pytest.mark.parametrize("nranks", (2, 3))
@pytest.mark.parametrize("scheme", ("mmc", "lf"))
@pytest.mark.parametrize("prec", (0, 1))
@pytest.mark.parametrize("name", sorted(CASES))
def test_partitioned_steps_equal_the_single_pool(gpulib, name, prec, scheme, nranks):
    from paper_1204_5849_gb300 import Partition, Pool
    mk_mesh, mk_state = CASES[name]
    mesh = mk_mesh()
    U0 = mk_state(mesh)
    params = _params(name, scheme)
    ref = Pool(mesh, prec)
    ref.write_leaves(U0)
    parts = [Partition(mesh, nranks, r) for r in range(nranks)]
    pools = []
    for part in parts:
        pool = Pool(mesh, prec)
        local = np.full_like(U0, np.nan)
        local[part.own] = U0[part.own]
        pool.write_leaves(local)
        pool.set_active(part.own)
        pools.append(pool)
    for step in range(3):
        assert _exchange(pools, parts, prec) > 0
        ref.fill_ghosts()
        dt_ref = ref.cfl_dt(params)
        ref.step(params)
        alphas = []
        for pool in pools:
            pool.fill_ghosts()
            alphas.append(pool.local_alpha(params))
        ag = np.max(np.stack(alphas), axis=0)                # the all-reduce (max)
        assert ag[0] == ref.speeds()[0][4]                   # alpha_g bitwise
        for pool in pools:
            pool.set_alpha(params, ag)
            assert pool.speeds()[0][0] == dt_ref[0]          # dt bitwise
            pool.step(params)
    R = ref.read_leaves()
    total = np.zeros(9)
    for pool, part in zip(pools, parts):
        G = pool.read_leaves()
        np.testing.assert_array_equal(G[part.own], R[part.own])
        total += pool.conservation()[0]
        assert pool.check() == 0
    want = ref.conservation()[0]
    np.testing.assert_allclose(total, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())
    for pool in pools:
        pool.close()
    ref.close()


def test_partitioned_pool_refuses_what_needs_exchanges_inside_a_step(gpulib):
    from paper_1204_5849_gb300 import MAP_FP64, MapError, Partition, Pool
    mesh = w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.OUTFLOW)   # mixed levels
    assert len({lv for (_, lv, _, _, _) in mesh.leaves}) > 1
    U0 = w.evaluate_on_mesh(mesh, rotor)
    part = Partition(mesh, 2, 0)
    pool = Pool(mesh, MAP_FP64)
    pool.write_leaves(U0)
    pool.set_active(part.own)
    p = dict(gamma=1.4, c_cfl=0.4, scheme="lf", limiter="minmod", reflux=0)
    pool.fill_ghosts()
    pool.set_alpha(p, pool.local_alpha(p))
    for bad, code in ((dict(scheme="weno"), -7), (dict(reflux=1), -7),
                      (dict(conduction="isotropic", kappa0=1e-3), -7)):
        with pytest.raises(MapError) as ei:
            pool.step(dict(p, **bad))
        assert ei.value.code == code, bad
    with pytest.raises(MapError) as ei:
        pool.advance(p, 1)
    assert ei.value.code == -8                               # MAP_ESTATE
    with pytest.raises(MapError):
        pool.set_active([0, 0])                              # repeated leaf
    pool.set_active(None)                                    # all leaves again: advance works
    pool.advance(p, 1)
    assert pool.check() == 0
    pool.close()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _proc(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_1204_5849_gb300 import MAP_FP32_FIX64, Partition, Pool
        mesh = w.uniform_mesh(3, 16, (2, 2, 1))
        U0 = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, amp=1e-2)
        params = dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="vanleer", eglm=1)
        part = Partition(mesh, world, rank)
        pool = Pool(mesh, MAP_FP32_FIX64)
        local = np.full_like(U0, np.nan)
        local[part.own] = U0[part.own]
        pool.write_leaves(local)
        pool.set_active(part.own)
        got = 0
        for _ in range(2):
            got += part.exchange(pool, dist, "cpu")
            pool.fill_ghosts()
            a = torch.from_numpy(pool.local_alpha(params))
            dist.all_reduce(a, op=dist.ReduceOp.MAX)
            pool.set_alpha(params, a.numpy())
            pool.step(params)
        G = pool.read_leaves()
        q.put((rank, part.own.tolist(), G[part.own], pool.speeds()[0][0], got, pool.check()))
        pool.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_through_gloo_on_one_gpu(gpulib):
    """Partition.exchange (map_pack_leaves, host copies through gloo, map_unpack_leaves) and
    the all-reduce of alpha_g between two processes, each with its own pool on cuda:0;
    their own leaves equal one pool's after two steps."""
    import torch.multiprocessing as mp
    from paper_1204_5849_gb300 import MAP_FP32_FIX64, Pool
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_proc, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    mesh = w.uniform_mesh(3, 16, (2, 2, 1))
    U0 = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, amp=1e-2)
    params = dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="vanleer", eglm=1)
    ref = Pool(mesh, MAP_FP32_FIX64)
    ref.write_leaves(U0)
    for _ in range(2):
        ref.fill_ghosts()
        ref.cfl_dt(params)
        ref.step(params)
    R = ref.read_leaves()
    for rank, own, G, dt, got, chk in res:
        np.testing.assert_array_equal(G, R[own])
        assert dt == ref.speeds()[0][0]
        assert got > 0 and chk == 0
    ref.close()
