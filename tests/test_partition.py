"""The partition over processes (Sec. 4.2 load balance, Sec. 4.3 boundary conditions between
processes), on the CPU: the library's host planner (map_plan_partition) and a halo
exchange between gloo ranks, checked against the single-process ghost fill and step of the
oracle, bitwise.

Each rank holds only its own leaves' interiors (every other leaf is NaN), receives from its
peers exactly the leaves the plan says it needs, fills its ghosts and steps with the oracle.
Its own leaves must then hold bitwise what one process holding everything computes: a leaf
missing from the plan would leak a NaN into them.
"""

from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import workloads as w
from workloads.problems import ensemble_problem, harris_sheet, rotor


def _meshes():
    return {
        "2d_periodic": w.uniform_mesh(2, 16, (4, 3)),
        "3d_periodic": w.uniform_mesh(3, 8, (3, 2, 2)),
        "2d_amr_outflow": w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.OUTFLOW),
        "3d_amr_slab": w.slab_amr_mesh(3, 8, (2, 2, 2), 1, half_widths=(0.08,)),
        "2d_amr_periodic": w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.PERIODIC,
                                             lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0)),
    }


def _state(name, mesh):
    if name.startswith("3d_amr"):
        return w.evaluate_on_mesh(mesh, harris_sheet)
    if name == "2d_amr_outflow":
        return w.evaluate_on_mesh(mesh, rotor)
    if mesh.ndim == 3:
        return w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, amp=1e-2)
    return w.evaluate_on_mesh(mesh, lambda X, Y, Z, **_: ensemble_problem(X, Y, Z, seed=7))


def _morton_order(mesh):
    """Leaves in the order the library numbers them: problem, then the bits of the lower
    corner's coordinates at the finest level interleaved (x lowest)."""
    top = max(lv for (_, lv, _, _, _) in mesh.leaves)

    def key(t):
        p, lv, i, j, k = t
        s = top - lv
        c = (i << s, j << s, k << s)
        m = 0
        for bit in range(21):
            for d in range(mesh.ndim):
                m |= ((c[d] >> bit) & 1) << (mesh.ndim * bit + d)
        return (p, m)
    return sorted(range(mesh.nleaves), key=lambda q: key(tuple(mesh.leaves[q][:5])))


@pytest.mark.parametrize("nranks", (1, 2, 3, 5))
@pytest.mark.parametrize("name", sorted(_meshes()))
def test_plan_is_equal_count_morton_ranges(name, nranks):
    from paper_1204_5849_gb300 import Partition, plan_partition
    mesh = _meshes()[name]
    owner, need = plan_partition(mesh, nranks)
    order = _morton_order(mesh)
    along = owner[order]
    assert np.all(np.diff(along) >= 0)                 # contiguous ranges along the curve
    counts = np.bincount(owner, minlength=nranks)
    n = mesh.nleaves
    assert counts.tolist() == [n * (r + 1) // nranks - n * r // nranks for r in range(nranks)]
    for r in range(nranks):
        assert np.all(need[r][owner == r] == 1)         # own leaves are needed
    if nranks == 1:
        assert np.all(need == 1)
    # what a rank receives from a peer is what that peer sends to it
    parts = [Partition(mesh, nranks, r) for r in range(nranks)]
    for r in range(nranks):
        for q in range(nranks):
            if q != r:
                np.testing.assert_array_equal(parts[r].recvs(q), parts[q].sends(r))


@pytest.mark.parametrize("name", sorted(_meshes()))
def test_plan_closure_covers_every_ghost_fill(name):
    """For 2..13 processes, in one process: a state that holds only what the plan says a
    process needs (NaN elsewhere) gives its own leaves, after the oracle's ghost fill,
    bitwise the ghosts of the full state."""
    from oracle import Oracle
    from paper_1204_5849_gb300 import plan_partition
    mesh = _meshes()[name]
    U = _state(name, mesh)
    ref = Oracle(mesh, U)
    ref.fill_ghosts()
    R = [ref.get_ghosted(b) for b in range(mesh.nleaves)]
    for nranks in (2, 3, 4, 5, 7, 13):
        if nranks > mesh.nleaves:
            continue
        owner, need = plan_partition(mesh, nranks)
        for r in range(nranks):
            local = np.where(need[r][:, None, None, None, None] != 0, U, np.nan)
            o = Oracle(mesh, local)
            o.fill_ghosts()
            for b in np.flatnonzero(owner == r):
                np.testing.assert_array_equal(o.get_ghosted(int(b)), R[int(b)], err_msg=f"{nranks} {r} {b}")


def test_plan_halo_is_a_thin_shell():
    """A periodic box of 4^3 blocks of 8^3 cut in two along the curve: each half needs one
    layer of blocks from the other (the ghost layers are 2 cells deep, a block 8), those
    next to the two faces of the cut (periodic), not the whole other half."""
    from paper_1204_5849_gb300 import plan_partition
    mesh = w.uniform_mesh(3, 8, (4, 4, 4))
    owner, need = plan_partition(mesh, 2)
    for r in range(2):
        halo = int(need[r].sum()) - int((owner == r).sum())
        assert 0 < halo <= 2 * 16 + 4 * 4, halo


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, name, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import Oracle
        from paper_1204_5849_gb300 import Partition
        mesh = _meshes()[name]
        U = _state(name, mesh)
        part = Partition(mesh, world, rank)
        # this process holds its own leaves only
        local = np.full_like(U, np.nan)
        local[part.own] = U[part.own]
        ops, inbox = [], []
        for peer in range(world):
            if peer == rank:
                continue
            snd, rcv = part.sends(peer), part.recvs(peer)
            if len(snd):
                ops.append(dist.P2POp(dist.isend, torch.from_numpy(np.ascontiguousarray(local[snd])), peer))
            if len(rcv):
                buf = torch.empty((len(rcv),) + U.shape[1:], dtype=torch.float64)
                ops.append(dist.P2POp(dist.irecv, buf, peer))
                inbox.append((rcv, buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for rcv, buf in inbox:
            local[rcv] = buf.numpy()
        received = sum(len(r) for r, _ in inbox)
        # the ghost fill and one step (fixed dt and c_h: the reduction is a separate
        # all-reduce) on this process against one process holding everything
        params = dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="minmod", eglm=1, eta=0.0,
                      dt_override=1e-3, ch_mode="fixed", ch=1.5, reflux=0)
        ref = Oracle(mesh, U)
        ref.fill_ghosts()
        mine = Oracle(mesh, local)
        mine.fill_ghosts()
        fill_ok = all(np.array_equal(mine.get_ghosted(int(b)), ref.get_ghosted(int(b))) for b in part.own)
        ref.cfl(params)
        ref.step(params)
        mine.cfl(params)
        mine.step(params)                               # the NaN leaves stay NaN
        step_ok = bool(np.array_equal(mine.get_state()[part.own], ref.get_state()[part.own]))
        q.put((rank, fill_ok, step_ok, received, len(part.own)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", (2, 3))
@pytest.mark.parametrize("name", sorted(_meshes()))
def test_gloo_halo_exchange_matches_single_process(name, world):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    mesh = _meshes()[name]
    assert sum(g[4] for g in got) == mesh.nleaves
    for rank, fill_ok, step_ok, received, nown in got:
        assert fill_ok, (name, rank)
        assert step_ok, (name, rank)
        assert received > 0


def test_plan_rejects_bad_input():
    from paper_1204_5849_gb300 import MapError, plan_partition
    mesh = w.uniform_mesh(2, 16, (2, 2))
    with pytest.raises(MapError) as ei:
        plan_partition(mesh, 0)
    assert ei.value.code == -1
    bad = w.uniform_mesh(2, 16, (2, 2))
    bad.leaves = bad.leaves[:3]                        # a hole in the domain
    with pytest.raises(MapError) as ej:
        plan_partition(bad, 2)
    assert ej.value.code == -1


def test_more_processes_than_leaves_leaves_some_idle():
    """Equal-count ranges with more processes than leaves: the first n processes own one
    leaf each, the rest none (and need nothing)."""
    from paper_1204_5849_gb300 import plan_partition
    mesh = w.uniform_mesh(2, 16, (2, 2))
    owner, need = plan_partition(mesh, 6)
    counts = np.bincount(owner, minlength=6)
    assert sorted(counts.tolist()) == [0, 0, 1, 1, 1, 1]
    for r in range(6):
        if counts[r] == 0:
            assert need[r].sum() == 0
