"""The oracle's flop counter, which gives the roofline its algorithmic flops per cell-update.

The counting build adds every floating-point operation the oracle executes to one of three
counters (ring-cell work, per-face work evaluated from both sides of each face, interior
work).  These tests pin the split by how each counter must scale with the block size and
the block count, so a loop filed under the wrong counter, or a face counted the wrong
number of times, changes a result here.
"""

from __future__ import annotations

import ctypes as C
import math

import numpy as np
import pytest

import workloads as w
from oracle import oracle as O

MINMOD_LF = dict(scheme="lf", limiter="minmod")


def _state(mesh):
    if mesh.ndim == 2:
        return w.evaluate_on_mesh(mesh, w.problems.ensemble_problem, seed=3)
    return w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3, amp=0.1)


def _count(mesh, params):
    return O.count_step_flops(mesh, _state(mesh), params)


def test_normal_build_has_no_counters():
    out = (C.c_ulonglong * 3)()
    assert O.lib().orc_flop_counts(out, 0) == 0
    assert list(out) == [0, 0, 0]


@pytest.mark.parametrize("ndim", [2, 3])
def test_counters_scale_as_their_regions(ndim):
    """Ring work scales with (nb+2)^d per block, face and cell work with nb^d; with minmod
    the count does not depend on the data, so per-region figures agree across meshes."""
    meshes = [w.uniform_mesh(ndim, 8, (2,) * ndim), w.uniform_mesh(ndim, 16, (1,) * ndim),
              w.uniform_mesh(ndim, 16, (3, 1, 2)[:ndim])]
    r8, r16, r16b = (_count(m, MINMOD_LF) for m in meshes)
    for r, m in zip((r8, r16, r16b), meshes):
        nb, nblk = m.nb, m.nleaves
        r["ring_per"] = r["ring"] / (nblk * (nb + 2) ** ndim)
        r["face_per"] = r["face"] / (2 * ndim * nblk * nb ** ndim)
        r["cell_per"] = r["cell"] / (nblk * nb ** ndim)
    for key in ("ring_per", "face_per", "cell_per"):
        assert r8[key] == r16[key] == r16b[key], key
        assert r8[key] == int(r8[key]), key          # whole operations per region unit
    assert math.isclose(r8["per_cell_update"], r16["per_cell_update"])


def test_face_work_is_one_lf_flux_per_face_plus_face_states():
    """Per face: the two reconstructed face states (4 operations per variable) and one
    Lax-Friedrichs flux, whose own count is read from the counter on a single call."""
    L = O.flop_lib()
    out = (C.c_ulonglong * 3)()
    L.orc_flop_counts(out, 1)
    a = np.array([1.0, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 2.0, 0.01])
    b = a * 1.01
    f = np.zeros(9)
    L.orc_lf_flux(0, O._dp(a), O._dp(b), 5 / 3, 1.0, O._dp(f))
    L.orc_flop_counts(out, 1)
    lf = sum(out)
    mesh = w.uniform_mesh(3, 8, (1, 1, 1))
    r = _count(mesh, MINMOD_LF)
    assert r["face"] / (2 * 3 * 8 ** 3) == lf + 4 * 9


def test_van_leer_adds_between_one_and_five_per_limiter_call():
    mesh = w.uniform_mesh(3, 8, (2, 1, 1))
    mm = _count(mesh, MINMOD_LF)
    vl = _count(mesh, dict(scheme="lf", limiter="vanleer"))
    calls = 3 * 9 * mesh.nleaves * (8 + 2) ** 3       # one slope per variable, dimension, ring cell
    extra = vl["ring"] - mm["ring"]
    assert calls <= extra <= 5 * calls
    assert vl["face"] == mm["face"] and vl["cell"] == mm["cell"]


def test_resistivity_adds_only_ring_and_cell_work():
    mesh = w.uniform_mesh(3, 8, (1, 1, 1))
    r0 = _count(mesh, MINMOD_LF)
    r1 = _count(mesh, dict(MINMOD_LF, eta=1e-3))
    assert r1["face"] == r0["face"]
    assert r1["ring"] > r0["ring"] and r1["cell"] > r0["cell"]


def test_weno_two_stages_and_no_ring_work():
    mesh = w.uniform_mesh(2, 8, (2, 2))
    r = _count(mesh, dict(scheme="weno"))
    assert r["ring"] == 0
    # two right-hand sides: the face counter holds 2 stages x 2 sides x ndim faces per cell
    per_face = r["face"] / (2 * 2 * 2 * mesh.nleaves * 64)
    assert per_face == int(per_face)


def test_bench_constant_matches_count_on_its_workload():
    """The benchmark's flops per cell-update: the count on the 64^3 version of its initial
    state (same blocks, scheme and limiter) lies within 0.5% of the stored 256^3 figure."""
    import bench
    from workloads.problems import config_alfven3d
    cfg = config_alfven3d()
    mesh = w.uniform_mesh(3, 16, (4, 4, 4))
    U0 = w.evaluate_on_mesh(mesh, w.alfven_wave, ndim=3)
    r = O.count_step_flops(mesh, U0, cfg["params"])
    assert abs(r["per_cell_update"] - bench.FLOPS_PER_CELL) <= 0.005 * bench.FLOPS_PER_CELL
