"""The allocation-free CFL entry point (map_cfl_dt_noalloc) against map_cfl_dt.

map_cfl_dt_noalloc is for callers that cannot allocate device memory (device memory owned by
another allocator, loops that must not synchronise the way cudaMalloc/cudaFree may): it
takes a state that already lives on the device and keeps its scratch in a static device
array.  Its results must equal the pool entry point's on the same state, call after call,
and the calls must allocate nothing.  This file is collected last so that a
stop-at-first-failure run has already run every other test.
"""

from __future__ import annotations

import gc

import numpy as np
import pytest

import workloads as w
from workloads.problems import ensemble_initial

pytestmark = pytest.mark.gpu


def padded_device_state(mesh, U, dtype):
    """The pool layout [block][9][nz+4][nb+4][nb+4] (2D: one z plane) on cuda:0."""
    import torch
    nb = mesh.nb
    n = mesh.nleaves
    NP = nb + 4
    NZ = NP if mesh.ndim == 3 else 1
    host = np.zeros((n, 9, NZ, NP, NP), dtype=np.float64)
    if mesh.ndim == 3:
        host[:, :, 2:2 + nb, 2:2 + nb, 2:2 + nb] = U
    else:
        host[:, :, 0:1, 2:2 + nb, 2:2 + nb] = U
    return torch.tensor(host.astype(dtype), device="cuda:0")


CASES = [
    ("fp64_3d_lf", 0, lambda: w.uniform_mesh(3, 16, (2, 2, 2)),
     lambda m: w.evaluate_on_mesh(m, w.alfven_wave, ndim=3, amp=1e-3),
     dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="vanleer")),
    ("fp32_2d_mmc", 1, lambda: w.ensemble_mesh(16, [64]),
     lambda m: ensemble_initial(m),
     dict(gamma=5 / 3, c_cfl=0.4, scheme="mmc", limiter="minmod")),
    ("fp64_3d_resistive_nb8", 0, lambda: w.uniform_mesh(3, 8, (2, 2, 2), lo=(-0.5, -0.5, -0.5),
                                                        hi=(0.5, 0.5, 0.5)),
     lambda m: w.evaluate_on_mesh(m, w.harris_sheet),
     dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="minmod", eta=1e-3)),
    ("fp32_2d_nb8_resistive", 1, lambda: w.uniform_mesh(2, 8, (3, 2)),
     lambda m: w.evaluate_on_mesh(m, w.orszag_tang),
     dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="vanleer", eta=2e-3)),
]


@pytest.mark.parametrize("name,prec,mk_mesh,mk_state,params", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_pool_entry_point(gpulib, name, prec, mk_mesh, mk_state, params):
    import torch
    from paper_1204_5849_gb300 import Pool
    from paper_1204_5849_gb300.binding import cfl_dt_noalloc

    mesh = mk_mesh()
    U = mk_state(mesh)
    pool = Pool(mesh, prec)
    pool.write_leaves(U)
    dt_ref = pool.cfl_dt(params)
    ref = pool.speeds()[0]            # dt, c_h, c_p, damping, alpha_g
    assert dt_ref[0] == ref[0]
    pool.close()

    dev = padded_device_state(mesh, U, np.float64 if prec == 0 else np.float32)
    torch.cuda.synchronize()
    dx = mesh.leaf_dx(0)
    # on a side stream of torch's (the call runs on and synchronises the stream it is given)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    out = cfl_dt_noalloc(dev.data_ptr(), prec, mesh.ndim, mesh.nb, mesh.nleaves, dx, params,
                         stream=side.cuda_stream)
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0.0)
    # the calls allocate nothing: neither torch's allocator nor the device's free memory moves
    # (the garbage collector is held off so that no unrelated tensor is freed meanwhile)
    gc.collect()
    torch.cuda.synchronize()
    gc.disable()
    try:
        alloc0 = torch.cuda.memory_allocated()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):            # two calls in a row share the static scratch
            out = cfl_dt_noalloc(dev.data_ptr(), prec, mesh.ndim, mesh.nb, mesh.nleaves, dx, params,
                                 stream=side.cuda_stream)
            np.testing.assert_allclose(out, ref, rtol=1e-12, atol=0.0)
            assert out[4] == ref[4]   # alpha_g: a maximum, exact
            assert torch.cuda.memory_allocated() == alloc0
            assert torch.cuda.mem_get_info()[0] == free0
    finally:
        gc.enable()


def test_noalloc_rejects_too_many_blocks(gpulib):
    import torch
    from paper_1204_5849_gb300 import MapError
    from paper_1204_5849_gb300.binding import NOALLOC_MAX_BLOCKS, cfl_dt_noalloc
    dev = torch.zeros(16, device="cuda:0", dtype=torch.float64)
    with pytest.raises(MapError) as ei:
        cfl_dt_noalloc(dev.data_ptr(), 0, 3, 16, NOALLOC_MAX_BLOCKS + 1, [0.1, 0.1, 0.1],
                       dict(gamma=5 / 3, c_cfl=0.4))
    assert ei.value.code == -1
    assert "MAP_NOALLOC_MAX_BLOCKS" in str(ei.value)


@pytest.mark.parametrize("bad", [dict(c_d=1.5), dict(c_d=0.0), dict(eta=-1e-3),
                                 dict(conduction="isotropic", kappa0=1e-3), dict(gamma=1.0)],
                         ids=["c_d_above_1", "c_d_zero", "eta_negative", "conduction", "gamma"])
def test_noalloc_rejects_what_the_pool_entry_point_rejects(gpulib, bad):
    """The parameter checks of map_cfl_dt, and thermal conduction, whose dt bound the
    allocation-free reduction does not compute."""
    from paper_1204_5849_gb300 import MapError
    from paper_1204_5849_gb300.binding import cfl_dt_noalloc
    mesh = w.uniform_mesh(2, 16, (2, 2))
    dev = padded_device_state(mesh, w.evaluate_on_mesh(mesh, w.orszag_tang), np.float64)
    params = dict(dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="minmod"), **bad)
    with pytest.raises(MapError) as ei:
        cfl_dt_noalloc(dev.data_ptr(), 0, 2, 16, mesh.nleaves, mesh.leaf_dx(0), params)
    assert ei.value.code == -1


@pytest.mark.parametrize("prec", (0, 1))
def test_noalloc_nan_state_is_rejected_like_the_pool(gpulib, prec):
    """A NaN cell (host input) gives MAP_ENONFINITE from both CFL entry points."""
    from paper_1204_5849_gb300 import MapError, Pool
    from paper_1204_5849_gb300.binding import cfl_dt_noalloc
    mesh = w.uniform_mesh(2, 16, (2, 2))
    U = w.evaluate_on_mesh(mesh, w.orszag_tang)
    U[2, 4, 0, 5, 9] = np.nan
    params = dict(gamma=5 / 3, c_cfl=0.4, scheme="lf", limiter="minmod")
    pool = Pool(mesh, prec)
    pool.write_leaves(U)
    with pytest.raises(MapError) as e1:
        pool.cfl_dt(params)
    pool.close()
    dev = padded_device_state(mesh, U, np.float64 if prec == 0 else np.float32)
    with pytest.raises(MapError) as e2:
        cfl_dt_noalloc(dev.data_ptr(), prec, 2, 16, mesh.nleaves, mesh.leaf_dx(0), params)
    assert e1.value.code == e2.value.code == -4            # MAP_ENONFINITE
