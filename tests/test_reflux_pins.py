"""Oracle pins for reflux at coarse/fine faces (Sec. 4.2, boundary step (2)).

Without reflux a coarse leaf and the fine leaves across a face each update with their own
flux through that face, so the totals of the conserved variables drift; with it the face
carries one flux on both sides.  Pinned here against what the method fixes:
* with every source switched off (EGLM sources off, no psi damping, no resistivity) on a
  periodic AMR mesh, the totals of all nine variables hold to round-off under MMC, LF and
  WENO in 2D and 3D, while without reflux they drift by orders of magnitude more;
* on a single-level mesh reflux changes nothing, bit for bit;
* only coarse cells next to a coarse/fine face change, and a uniform state stays uniform.
"""

from __future__ import annotations

import numpy as np
import pytest

import workloads as w
from oracle import Oracle

FLUX_ONLY = dict(eglm=0, cp_mode="fixed", cp=0.0, eta=0.0)


def _amr(ndim):
    if ndim == 2:
        return w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.PERIODIC,
                                 lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0))
    return w.radial_amr_mesh(3, 8, (4, 4, 4), 1, radii=(0.2,), bc=w.mesh.PERIODIC,
                             lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0.5))


def _state(mesh):
    return w.evaluate_on_mesh(mesh, w.problems.ensemble_problem, seed=5)


def _drift(mesh, U0, params, steps):
    o = Oracle(mesh, U0)
    s0 = o.conservation()
    o.advance(params, steps)
    s1 = o.conservation()
    return (np.abs(s1 - s0) / np.maximum(np.abs(s0), 1e-3)).max()


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme", ["mmc", "lf", "weno"])
def test_reflux_conserves_every_variable(ndim, scheme):
    mesh = _amr(ndim)
    assert len(set(mesh.leaves[:, 1].tolist())) > 1
    U0 = _state(mesh)
    p = dict(FLUX_ONLY, scheme=scheme)
    with_rf = _drift(mesh, U0, dict(p, reflux=1), 3)
    without = _drift(mesh, U0, dict(p, reflux=0), 3)
    assert with_rf <= 2e-14, with_rf
    assert without >= 1e-5, without


@pytest.mark.parametrize("scheme", ["mmc", "lf", "weno"])
def test_reflux_is_identity_on_a_single_level(scheme):
    mesh = w.uniform_mesh(2, 8, (3, 2))
    U0 = _state(mesh)
    out = []
    for rf in (0, 1):
        o = Oracle(mesh, U0)
        o.advance(dict(scheme=scheme, reflux=rf), 2)
        out.append(o.get_state())
    np.testing.assert_array_equal(out[0], out[1])


def _coarse_face_cells(mesh):
    """Per leaf a boolean mask of interior cells next to a face whose same-level neighbour
    is refined (brute force over the leaf list)."""
    nb, nd = mesh.nb, mesh.ndim
    leaves = {tuple(int(x) for x in r) for r in mesh.leaves}
    prob = mesh.problems[0]
    nz = nb if nd == 3 else 1
    masks = []
    for (p, L, i, j, k) in [tuple(int(x) for x in r) for r in mesh.leaves]:
        m = np.zeros((nz, nb, nb), dtype=bool)
        ijk = [i, j, k]
        for d in range(nd):
            n = prob.nbase[d] << L
            for side in (0, 1):
                c = list(ijk)
                c[d] = (c[d] + (1 if side else -1)) % n
                fine = any((p, L + 1, 2 * c[0] + a, 2 * c[1] + b, (2 * c[2] + e) if nd == 3 else 0) in leaves
                           for a in (0, 1) for b in (0, 1) for e in ((0, 1) if nd == 3 else (0,)))
                if not fine:
                    continue
                sl = [slice(None)] * 3
                sl[2 - d] = nb - 1 if side else 0
                m[tuple(sl)] = True
        masks.append(m)
    return np.array(masks)


@pytest.mark.parametrize("ndim", [2, 3])
def test_reflux_touches_only_coarse_cells_at_coarse_fine_faces(ndim):
    mesh = _amr(ndim)
    U0 = _state(mesh)
    out = []
    for rf in (0, 1):
        o = Oracle(mesh, U0)
        o.advance(dict(scheme="lf", reflux=rf), 1)
        out.append(o.get_state())
    changed = np.any(out[0] != out[1], axis=1)              # (leaf, z, y, x)
    expect = _coarse_face_cells(mesh)
    assert expect.any()
    assert not np.any(changed & ~expect)
    assert changed[expect].mean() > 0.9                      # nearly every such cell moves


def test_reflux_keeps_a_uniform_state_uniform():
    mesh = _amr(2)
    U0 = w.evaluate_on_mesh(mesh, w.problems.uniform_state)
    o = Oracle(mesh, U0)
    o.advance(dict(scheme="lf", reflux=1), 2)
    np.testing.assert_array_equal(o.get_state(), U0)
