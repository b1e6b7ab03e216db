"""Non-finite host input: a NaN or an infinity written into one cell of the state.

The Sec. 3.7 time step is built from the maximum signal speed over every leaf cell, so a
non-finite speed anywhere must reach the reduction's result: where the oracle's CFL returns
an error, so must both CFL entry points of the library (map_cfl_dt, map_cfl_dt_noalloc),
for every cell position (in particular every lane of a warp, not only the last), every
write path (map_write_leaves, map_write_leaves_async) and both precisions; a NaN always
does.  An infinite density gives that cell a zero, finite signal speed in the oracle and
in the library alike, and a NaN in psi enters no signal speed: the reductions then agree
that dt is finite, and the state checks after the step (oracle step status, map_check)
report the non-finite cell.  The pool recovers after a clean write.  These are host-side
inputs only: nothing here faults the GPU.
"""

from __future__ import annotations

import numpy as np
import pytest

import workloads as w
from oracle import Oracle

pytestmark = pytest.mark.gpu

ENONFINITE = -4
PARAMS = dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="vanleer", eglm=1)

MESHES = {
    "2d16": lambda: w.uniform_mesh(2, 16, (2, 2)),
    "3d16": lambda: w.uniform_mesh(3, 16, (2, 1, 1)),
    "3d8": lambda: w.uniform_mesh(3, 8, (2, 2, 1)),
}

# (block, variable, z, y, x): x + nb y runs over several lanes of a warp (0, 5, 17, 31 ...)
POSITIONS = {
    "2d16": [(0, 0, 0, 0, 0), (1, 1, 0, 0, 5), (2, 7, 0, 1, 1), (3, 4, 0, 1, 15), (3, 6, 0, 9, 7)],
    "3d16": [(0, 0, 0, 0, 0), (1, 2, 3, 1, 9), (0, 7, 15, 15, 15), (1, 5, 7, 1, 15)],
    "3d8": [(0, 0, 0, 0, 0), (1, 3, 2, 1, 7), (2, 7, 7, 3, 7), (3, 4, 4, 2, 5)],
}


def _state(mesh):
    return w.evaluate_on_mesh(mesh, w.orszag_tang) if mesh.ndim == 2 else \
        w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, amp=1e-2)


def _write(pool, U, how):
    import torch
    if how == "sync":
        pool.write_leaves(U)
    else:
        pinned = torch.empty(U.shape, dtype=torch.float64, pin_memory=True)
        pinned.numpy()[...] = U
        pool.write_leaves_async_ptr(pinned.data_ptr())
        torch.cuda.synchronize()


def _padded(mesh, U, prec):
    import torch
    nb, NP = mesh.nb, mesh.nb + 4
    NZ = NP if mesh.ndim == 3 else 1
    host = np.zeros((mesh.nleaves, 9, NZ, NP, NP))
    if mesh.ndim == 3:
        host[:, :, 2:2 + nb, 2:2 + nb, 2:2 + nb] = U
    else:
        host[:, :, 0:1, 2:2 + nb, 2:2 + nb] = U
    return torch.tensor(host.astype(np.float64 if prec == 0 else np.float32), device="cuda:0")


@pytest.mark.parametrize("how", ("sync", "async"))
@pytest.mark.parametrize("bad", (np.nan, np.inf, -np.inf), ids=("nan", "inf", "-inf"))
@pytest.mark.parametrize("prec", (0, 1))
@pytest.mark.parametrize("geom", tuple(MESHES))
def test_nonfinite_cell_rejected_by_every_cfl(gpulib, geom, prec, bad, how):
    from paper_1204_5849_gb300 import MapError, Pool
    from paper_1204_5849_gb300.binding import cfl_dt_noalloc
    mesh = MESHES[geom]()
    U0 = _state(mesh)
    pool = Pool(mesh, prec)
    _write(pool, U0, how)
    dt_clean = pool.cfl_dt(PARAMS)
    rejected = 0
    for (b, v, z, y, x) in POSITIONS[geom]:
        where = (b, v, z, y, x)
        U = U0.copy()
        U[b, v, z, y, x] = bad
        # the oracle's decision
        orc = Oracle(mesh, U)
        orc.fill_ghosts()
        dto = orc.cfl(PARAMS)
        orc_rejects = orc._rc == -2
        if np.isnan(bad):
            assert orc_rejects, where
        rejected += orc_rejects
        # the pool entry point decides the same
        _write(pool, U, how)
        if orc_rejects:
            with pytest.raises(MapError) as ei:
                pool.cfl_dt(PARAMS)
            assert ei.value.code == ENONFINITE, where
        else:
            dtp = pool.cfl_dt(PARAMS)
            if prec == 0:
                assert dtp[0] == dto[0], where
            # the step then reports the non-finite cell, as the oracle's step does
            assert orc.step(PARAMS) == -2, where
            pool.fill_ghosts()
            pool.step(PARAMS)
            assert pool.check() == ENONFINITE, where
        # the allocation-free entry point on the same state
        dev = _padded(mesh, U, prec)
        if orc_rejects:
            with pytest.raises(MapError) as ej:
                cfl_dt_noalloc(dev.data_ptr(), prec, mesh.ndim, mesh.nb, mesh.nleaves, mesh.leaf_dx(0), PARAMS)
            assert ej.value.code == ENONFINITE, where
        else:
            out = cfl_dt_noalloc(dev.data_ptr(), prec, mesh.ndim, mesh.nb, mesh.nleaves, mesh.leaf_dx(0), PARAMS)
            assert np.isfinite(out[0]) and out[0] > 0, where
        # the pool recovers after a clean write
        _write(pool, U0, how)
        assert pool.cfl_dt(PARAMS)[0] == dt_clean[0]
    # every kind of bad value is rejected by the reduction somewhere (momentum, field, energy)
    assert rejected >= 2
    pool.advance(PARAMS, 1)
    assert pool.check() == 0
    pool.close()


@pytest.mark.parametrize("prec", (0, 1))
@pytest.mark.parametrize("geom", ("2d16", "3d16"))
def test_nan_in_psi_caught_after_the_step(gpulib, geom, prec):
    """psi enters no signal speed: the reductions agree that dt is the clean state's, and
    the state check after one step reports the non-finite cell (oracle step -2,
    map_check MAP_ENONFINITE) for the plain and the graph-replayed step alike."""
    from paper_1204_5849_gb300 import Pool
    from paper_1204_5849_gb300.binding import cfl_dt_noalloc
    mesh = MESHES[geom]()
    U0 = _state(mesh)
    U = U0.copy()
    U[1, 8, 0, 3, 6] = np.nan
    orc = Oracle(mesh, U)
    orc.fill_ghosts()
    dto = orc.cfl(PARAMS)
    assert orc._rc == 0
    assert orc.step(PARAMS) == -2
    pool = Pool(mesh, prec)
    pool.write_leaves(U0)
    dt_clean = pool.cfl_dt(PARAMS)
    pool.write_leaves(U)
    assert pool.cfl_dt(PARAMS)[0] == dt_clean[0]
    if prec == 0:
        assert dt_clean[0] == dto[0]
    out = cfl_dt_noalloc(_padded(mesh, U, prec).data_ptr(), prec, mesh.ndim, mesh.nb, mesh.nleaves,
                         mesh.leaf_dx(0), PARAMS)
    assert out[0] == dt_clean[0]
    pool.fill_ghosts()
    pool.step(PARAMS)
    assert pool.check() == ENONFINITE
    assert pool.check() == 0                      # map_check clears the error word
    pool.write_leaves(U)
    pool.advance(PARAMS, 1)
    assert pool.check() == ENONFINITE
    pool.write_leaves(U0)
    pool.advance(PARAMS, 2)
    assert pool.check() == 0
    pool.close()
