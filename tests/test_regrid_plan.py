"""The regrid decision (Sec. 4.5 refinement rule with 2:1 balance): oracle pins on CPU and
the library's plan against the oracle's on the GPU."""

from __future__ import annotations

import numpy as np
import pytest

import workloads as w
from oracle import Oracle
from oracle.oracle import plan_regrid


def _mesh(leaves, nbase=(2, 2, 1), ndim=2, bc=0):
    pr = w.Problem(tuple(nbase), bc=((bc, bc),) * 3)
    return w.Mesh(ndim, 8, [pr], np.asarray(leaves, dtype=np.int32).reshape(-1, 5))


def test_plan_refine_one_block_uniform():
    m = w.uniform_mesh(2, 8, (2, 2))
    flags = np.array([1, 0, 0, 0], dtype=np.int8)
    new = plan_regrid(m, flags, 3)
    want = [(0, 1, 0, 0, 0), (0, 1, 1, 0, 0), (0, 1, 0, 1, 0), (0, 1, 1, 1, 0),
            (0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0)]
    assert [tuple(r) for r in new] == want
    Oracle(w.Mesh(2, 8, m.problems, new))          # the result is a valid 2:1 tree


def test_plan_balance_propagates():
    # level-1 children in the lower-left quadrant, level-0 elsewhere (periodic 2x2 base)
    leaves = [(0, 1, a, b, 0) for b in (0, 1) for a in (0, 1)] + [(0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0)]
    m = _mesh(leaves)
    flags = np.zeros(len(leaves), dtype=np.int8)
    flags[3] = 1                                   # (1, 1, 1): touches all three level-0 blocks
    new = plan_regrid(m, flags, 3)
    levels = {tuple(r[2:4]) + (int(r[1]),) for r in new}
    # every level-0 block touching the new level-2 children had to become level 1
    assert not any(r[1] == 0 for r in new)
    assert sum(1 for r in new if r[1] == 2) == 4
    Oracle(w.Mesh(2, 8, m.problems, new))


def test_plan_coarsen_all_siblings_only():
    leaves = [(0, 1, a, b, 0) for b in (0, 1) for a in (0, 1)] + [(0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0)]
    m = _mesh(leaves)
    f = np.array([-1, -1, -1, -1, 0, 0, 0], dtype=np.int8)
    new = plan_regrid(m, f, 3)
    assert [tuple(r) for r in new] == [(0, 0, 0, 0, 0), (0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0)]
    f2 = f.copy()
    f2[2] = 0                                      # one sibling keeps: no coarsening
    assert [tuple(r) for r in plan_regrid(m, f2, 3)] == [tuple(r) for r in m.leaves]


def test_plan_coarsen_blocked_by_finer_neighbour():
    # base 4x2 (periodic x, outflow y): P = (1,0) refined to level 1; its neighbour N = (2,0)
    # refined to level 1 with N's child (4,0) refined again to level 2.  Coarsening P back to
    # level 0 would put level 0 next to those level-2 blocks, so it must not happen.
    P_children = [(0, 1, a, b, 0) for b in (0, 1) for a in (2, 3)]
    N_children = [(0, 1, 5, 0, 0), (0, 1, 4, 1, 0), (0, 1, 5, 1, 0)]
    N4_children = [(0, 2, 8 + a, b, 0) for b in (0, 1) for a in (0, 1)]
    coarse = [(0, 0, 0, 0, 0), (0, 0, 3, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0), (0, 0, 2, 1, 0), (0, 0, 3, 1, 0)]
    leaves = P_children + N_children + N4_children + coarse
    pr = w.Problem((4, 2, 1), bc=((0, 0), (1, 1), (0, 0)))
    m = w.Mesh(2, 8, [pr], np.asarray(leaves, dtype=np.int32))
    Oracle(m)                                       # a valid 2:1 tree
    f = np.zeros(len(leaves), dtype=np.int8)
    f[:4] = -1                                      # P's children want to coarsen
    new = plan_regrid(m, f, 3)
    assert [tuple(r) for r in new] == [tuple(r) for r in m.leaves]
    # with N's level-2 children flagged to coarsen as well, N's child coarsens this cycle and
    # P (whose neighbour was still refined below level 1 when the cycle began) the next one
    f[7:11] = -1
    new2 = plan_regrid(m, f, 3)
    t2 = [tuple(int(v) for v in r) for r in new2]
    assert (0, 1, 4, 0, 0) in t2 and (0, 0, 1, 0, 0) not in t2
    m2 = w.Mesh(2, 8, m.problems, new2)
    Oracle(m2)
    f2 = np.array([-1 if (r[1] == 1 and r[2] in (2, 3)) else 0 for r in new2], dtype=np.int8)
    t3 = [tuple(int(v) for v in r) for r in plan_regrid(m2, f2, 3)]
    assert (0, 0, 1, 0, 0) in t3
    Oracle(w.Mesh(2, 8, m.problems, np.asarray(t3, dtype=np.int32)))


@pytest.mark.gpu
@pytest.mark.parametrize("ndim", (2, 3))
def test_library_plan_matches_oracle(gpulib, ndim):
    from paper_1204_5849_gb300 import MAP_FP64, Pool
    if ndim == 2:
        m = w.radial_amr_mesh(2, 16, (4, 4), 2, radii=(0.12, 0.3), bc=w.mesh.OUTFLOW)
    else:
        m = w.slab_amr_mesh(3, 8, (4, 4, 4), 1, half_widths=(0.1,))
    rng = np.random.default_rng(7)
    pool = Pool(m, MAP_FP64)
    for trial in range(6):
        flags = rng.choice(np.array([-1, 0, 1], dtype=np.int8), size=m.nleaves, p=[0.5, 0.3, 0.2])
        want = plan_regrid(m, flags, 3)
        got = pool.plan_regrid(flags, 3)
        np.testing.assert_array_equal(got, want)


@pytest.mark.gpu
def test_adapt_cycle_matches_oracle(gpulib):
    """Flags -> plan -> regrid every 2 steps on the rotor (FP64): states stay in parity."""
    from paper_1204_5849_gb300 import MAP_FP64, Pool
    m = w.radial_amr_mesh(2, 16, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.OUTFLOW)
    U0 = w.evaluate_on_mesh(m, w.rotor)
    p = dict(gamma=1.4, c_cfl=0.4, scheme="weno", limiter="minmod", eglm=1)
    r = dict(vars=("rho", "p"), thr=0.2, coarsen=0.1, max_level=3)
    pool = Pool(m, MAP_FP64, max_blocks=4096)
    pool.write_leaves(U0)
    orc = Oracle(m, U0)
    mesh = m
    for cycle in range(3):
        for _ in range(2):
            pool.fill_ghosts(); pool.cfl_dt(p); pool.step(p)
            orc.fill_ghosts(); orc.cfl(p); orc.step(p)
        orc.fill_ghosts()
        f_o, _ = orc.flags(p, r)
        new = plan_regrid(mesh, f_o, r["max_level"])
        newmesh = w.Mesh(mesh.ndim, mesh.nb, mesh.problems, new)
        pmesh = pool.adapt(p, r)
        np.testing.assert_array_equal(pmesh.leaves, new)
        if not np.array_equal(new, mesh.leaves):
            orc = orc.regrid(newmesh)
        mesh = newmesh
        G, R = pool.read_leaves(), orc.get_state()
        for v in range(9):
            scale = max(float(np.abs(R[:, v]).max()), 1e-3)
            assert float(np.abs(G[:, v] - R[:, v]).max()) <= 1e-11 * scale
