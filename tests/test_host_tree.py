"""The block-tree logic of the library on the host, without a GPU (map_check_leaves,
map_plan_leaves): validation of leaf lists (Sec. 4.1: complete parents, covered domains, 2:1
over faces, edges and corners) with its reasons, on lists small enough for one host thread
and large enough for several; and the regrid decision (Sec. 4.5) leaf for leaf, in order,
against the oracle's brute-force planner, which is written independently over sets of block
keys, on random flags.
"""

from __future__ import annotations

import zlib
from dataclasses import replace

import numpy as np
import pytest

import workloads as w
from workloads.problems import CONFIGS
from oracle import Oracle
from oracle.oracle import plan_regrid as oracle_plan


def lib():
    from paper_1204_5849_gb300 import check_leaves, load, plan_leaves
    try:
        load()
    except Exception as e:                                   # the library is not built
        pytest.skip(f"libmapgb300.so not available: {e}")
    return check_leaves, plan_leaves


def _meshes():
    return {
        "uniform_3d": w.uniform_mesh(3, 8, (4, 4, 2)),
        "radial_2d_periodic": w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.PERIODIC,
                                                lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0)),
        "rotor_2d_outflow": CONFIGS["rotor_amr"]()["mesh"],          # 3028 leaves, 4 levels
        "harris_3d": CONFIGS["harris_amr"]()["mesh"],                # 9472 leaves, 3 levels
        "ensemble_2d": CONFIGS["ensemble"](small=True)["mesh"],      # several problems
    }


@pytest.mark.parametrize("name", list(_meshes()))
def test_valid_meshes_accepted(name):
    check_leaves, _ = lib()
    assert check_leaves(_meshes()[name]) == ""


def _refine_twice(leaves, c):
    i, j = c
    out = [tuple(r) for r in leaves if not (r[1] == 0 and (r[2], r[3]) == (i, j))]
    kids = [(0, 1, 2 * i + a, 2 * j + b, 0) for b in (0, 1) for a in (0, 1)]
    g = kids.pop(0)
    return out + kids + [(0, 2, 2 * g[2] + a, 2 * g[3] + b, 0) for b in (0, 1) for a in (0, 1)]


@pytest.mark.parametrize("n", [8, 64])                       # 64 blocks, or 4096 (several threads)
def test_invalid_trees_rejected_with_their_reason(n):
    check_leaves, _ = lib()
    mesh = w.uniform_mesh(2, 8, (n, n))
    leaves = [tuple(r) for r in mesh.leaves]
    cases = {
        "2:1 balance violated": _refine_twice(_refine_twice(leaves, (n - 3, n - 2)), (1, 2)),
        "duplicate leaf": leaves + [leaves[n + 3]],
        "domain not covered": leaves[:5] + leaves[6:],
        "incomplete parent": [r for r in _refine_twice(leaves, (2, 3)) if r != (0, 1, 5, 6, 0)],
        "leaf out of range": leaves + [(0, 0, n, 0, 0)],
    }
    for why, lv in cases.items():
        m = replace(mesh, leaves=np.array(lv, dtype=np.int32))
        got = check_leaves(m)
        assert why in got, (why, got)
        if why != "leaf out of range":
            with pytest.raises(ValueError):                  # the oracle rejects it as well
                Oracle(m, np.zeros((m.nleaves, 9, 1, 8, 8)))


def test_unbalanced_radial_mesh_rejected_by_both():
    check_leaves, _ = lib()
    m = w.radial_amr_mesh(2, 16, (4, 4), 2, radii=(0.2, 0.35))
    assert "2:1 balance violated" in check_leaves(m)
    with pytest.raises(ValueError):
        Oracle(m, np.zeros((m.nleaves, 9, 1, 16, 16)))


@pytest.mark.parametrize("name", list(_meshes()))
@pytest.mark.parametrize("mix", [(0.6, 0.3, 0.1), (0.2, 0.3, 0.5), (1 / 3, 1 / 3, 1 / 3)])
def test_plan_matches_the_oracle_planner(name, mix):
    check_leaves, plan_leaves = lib()
    mesh = _meshes()[name]
    rng = np.random.default_rng(zlib.crc32(f"{name}{mix}".encode()))
    for _ in range(3):
        flags = rng.choice(np.array([-1, 0, 1], dtype=np.int8), mesh.nleaves, p=list(mix))
        max_level = mesh.max_level + 1
        got = plan_leaves(mesh, flags, max_level)
        ref = np.asarray(oracle_plan(mesh, flags, max_level), dtype=np.int32)
        np.testing.assert_array_equal(got, ref)
        assert check_leaves(replace(mesh, leaves=got)) == ""
