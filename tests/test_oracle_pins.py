"""Pins of the FP64 CPU oracle against what the paper prints and what the mathematics fixes.

Each test names the passage it follows (sections/tables of Jiang, Fang & Chen,
arXiv:1204.5849).  None of these tests needs a GPU.
"""

from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest

import workloads as w
from workloads.problems import (advection_2d, alfven_wave, brio_wu, conserved_from_primitive,
                                divb_bump, ensemble_problem, field_loop, orszag_tang, uniform_state)
from oracle import Oracle
from oracle import oracle as O
from tests.helpers import (advection_1d, advection_strip, assemble_uniform, l1, quadratic_estimate,
                           run_to_time, two_level_mesh)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCHEMES = ("mmc", "lf", "weno")


def P(**kw):
    p = dict(gamma=5.0 / 3.0, c_cfl=0.4, scheme="mmc", limiter="minmod", eta=0.0, eglm=1)
    p.update(kw)
    return p


def to_global(mesh, U):
    return np.stack([assemble_uniform(mesh, U, v) for v in range(9)])


def from_global(mesh, G):
    nb = mesh.nb
    bz = nb if mesh.ndim == 3 else 1
    out = np.empty((mesh.nleaves, 9, bz, nb, nb))
    for b, (p, lv, i, j, k) in enumerate(mesh.leaves):
        out[b] = G[:, k * bz:(k + 1) * bz, j * nb:(j + 1) * nb, i * nb:(i + 1) * nb]
    return out


# --- 1. uniform state is unchanged bitwise (Equ:basic telescopes to zero) ---------------

@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("limiter", ("minmod", "vanleer"))
@pytest.mark.parametrize("ndim", (2, 3))
def test_uniform_state_bitwise(scheme, limiter, ndim):
    m = w.uniform_mesh(ndim, 8, (2, 2, 2))
    U0 = w.evaluate_on_mesh(m, uniform_state)
    o = Oracle(m, U0)
    p = P(scheme=scheme, limiter=limiter, eta=1e-3 if ndim == 3 else 0.0)
    for _ in range(2):
        o.fill_ghosts(); o.cfl(p); o.step(p)
    np.testing.assert_array_equal(o.get_state(), U0)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_uniform_state_bitwise_amr(scheme):
    m = w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.OUTFLOW)
    assert m.max_level == 2
    U0 = w.evaluate_on_mesh(m, uniform_state)
    o = Oracle(m, U0)
    p = P(scheme=scheme)
    for _ in range(2):
        o.fill_ghosts(); o.cfl(p); o.step(p)
    np.testing.assert_array_equal(o.get_state(), U0)


# --- 2. periodic conservation in GLM mode (Equ:basic is telescoping) ---------------------

@pytest.mark.parametrize("scheme,ndim,eta", [("mmc", 2, 0.0), ("lf", 2, 0.0), ("weno", 2, 0.0),
                                             ("lf", 3, 0.0), ("lf", 2, 2e-3), ("weno", 3, 1e-3)])
def test_periodic_conservation_glm(scheme, ndim, eta):
    if ndim == 2:
        m = w.uniform_mesh(2, 16, (2, 2))
        U0 = w.evaluate_on_mesh(m, orszag_tang)
    else:
        m = w.uniform_mesh(3, 8, (2, 2, 2))
        U0 = w.evaluate_on_mesh(m, alfven_wave, amp=0.05)
    o = Oracle(m, U0)
    p = P(scheme=scheme, limiter="vanleer" if scheme == "lf" else "minmod", eglm=0, eta=eta)
    s_prev = o.conservation()[0]
    for _ in range(3):
        o.fill_ghosts(); o.cfl(p)
        assert o.step(p) == 0
        s = o.conservation()[0]
        vol = np.prod(m.leaf_dx(0)[:ndim])
        scale = np.abs(o.get_state()).sum(axis=(0, 2, 3, 4)) * vol
        for v in range(8):  # rho, m, B, e (psi has its damping source)
            assert abs(s[v] - s_prev[v]) <= 1e-13 * max(scale[v], 1e-300), (v, s[v] - s_prev[v])
        s_prev = s


# --- 3. psi damping: one step multiplies psi by c_d (Sec. 2, c_p formula) ----------------

@pytest.mark.parametrize("scheme", SCHEMES)
def test_psi_only_damping(scheme):
    m = w.uniform_mesh(2, 8, (2, 2))
    U0 = w.evaluate_on_mesh(m, uniform_state, psi=0.37)
    o = Oracle(m, U0)
    p = P(scheme=scheme, c_d=0.18)
    o.fill_ghosts(); o.cfl(p); o.step(p)
    U = o.get_state()
    np.testing.assert_array_equal(U[:, :8], U0[:, :8])
    np.testing.assert_allclose(U[:, 8], 0.18 * 0.37, rtol=4e-16 * 4)


def test_speeds_closed_form():
    """alpha_g and dt for a uniform state with B along x: the fast speed is max(a, b_x)
    along B and sqrt(a^2 + b^2) across it (Sec. 3.7 dt formula)."""
    m = w.uniform_mesh(2, 8, (2, 2))
    gamma, rho, p0, bx, vx, vy = 5 / 3, 1.3, 0.7, 0.9, 0.4, -0.25
    U0 = w.evaluate_on_mesh(m, uniform_state, rho=rho, v=(vx, vy, 0.0), b=(bx, 0.0, 0.0), p=p0)
    o = Oracle(m, U0)
    dt = o.cfl(P(c_cfl=0.4))[0]
    a, b = math.sqrt(gamma * p0 / rho), bx / math.sqrt(rho)
    alpha_x = abs(vx) + max(a, b)
    alpha_y = abs(vy) + math.sqrt(a * a + b * b)
    ag = max(alpha_x, alpha_y)
    dx = 1.0 / 16
    assert dt == pytest.approx(0.4 * dx / (2 * ag), rel=1e-14)
    sp = o.speeds()[0]
    assert sp[1] == pytest.approx(ag, rel=1e-14)                        # c_h = alpha_g
    assert sp[3] == pytest.approx(0.18, rel=1e-14)                      # damping = c_d
    assert sp[2] == pytest.approx(math.sqrt(-dt * ag * ag / math.log(0.18)), rel=1e-14)


# --- 4. linear Alfven wave: second-order convergence to the closed form -----------------

def _alfven_error(ndim, n, scheme, T, limiter):
    nbk = n // 16
    m = w.uniform_mesh(ndim, 16, (nbk, nbk, nbk))
    amp = 1e-6
    o = Oracle(m, w.evaluate_on_mesh(m, alfven_wave, ndim=ndim, amp=amp))
    run_to_time(o, P(scheme=scheme, limiter=limiter), T)
    exact = w.evaluate_on_mesh(m, alfven_wave, ndim=ndim, amp=amp, t=T)
    U = o.get_state()
    comps = [6] if ndim == 2 else [5, 6]
    return sum(l1(U[:, c], exact[:, c]) for c in comps) / amp


@pytest.mark.parametrize("scheme,limiter", [("lf", "vanleer"), ("mmc", "minmod"), ("weno", "minmod")])
def test_alfven_2d_convergence(scheme, limiter):
    e = [_alfven_error(2, n, scheme, 0.5, limiter) for n in (32, 64, 128)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    # asymptotic order >= 1.7; the coarsest pair is limiter-clipped (the paper's own MMC
    # order at its coarsest pair in Table 2 is 1.59)
    assert orders[1] >= 1.7 and orders[0] >= 1.5, (e, orders)
    assert e[-1] < 0.05


def test_alfven_3d_convergence():
    e = [_alfven_error(3, n, "lf", 0.25, "vanleer") for n in (16, 32)]
    # 16^3 puts under 10 cells on a wavelength along the diagonal: coarse-pair order
    assert math.log2(e[0] / e[1]) >= 1.5, e


# --- 5. advection: the paper's Tables 1 and 2 -------------------------------------------

def _advect_1d(n, scheme):
    def ic(X, Y, Z, t=0.0, **_):
        rho = (np.sin(2 * math.pi * (X - t)) + 2) / 3
        return conserved_from_primitive(rho, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.4)
    m = w.uniform_mesh(2, 16, (n // 16, 1), lo=(-0.5, 0, 0), hi=(0.5, 16.0 / n, 1))
    o = Oracle(m, w.evaluate_on_mesh(m, ic))
    run_to_time(o, P(gamma=1.4, c_cfl=0.8, scheme=scheme), 1.0)
    return l1(o.get_state()[:, 0], w.evaluate_on_mesh(m, ic, t=1.0)[:, 0])


def _advect_2d(n, scheme):
    s3 = math.sqrt(3.0)
    m = w.uniform_mesh(2, 16, (n // 16, n // 16), lo=(-0.5, -s3 / 2, 0), hi=(0.5, s3 / 2, 1))
    o = Oracle(m, w.evaluate_on_mesh(m, advection_2d))
    run_to_time(o, P(gamma=1.4, scheme=scheme), 1.0)
    return l1(o.get_state()[:, 0], w.evaluate_on_mesh(m, advection_2d, t=1.0)[:, 0])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_table1_1d_advection(scheme):
    g = json.load(open(os.path.join(GOLDEN, "advection_tables.json")))["table1_1d"]
    e = [_advect_1d(n, scheme) for n in g["N"]]
    for got, want in zip(e, g[scheme]):
        assert 0.75 * want <= got <= 1.25 * want, (scheme, got, want)
    assert abs(math.log2(e[0] / e[1]) - g["order_128_256"][scheme]) <= 0.1


@pytest.mark.parametrize("scheme", SCHEMES)
def test_table2_2d_advection(scheme):
    g = json.load(open(os.path.join(GOLDEN, "advection_tables.json")))["table2_2d"]
    e = [_advect_2d(n, scheme) for n in g["N"]]
    for got, want in zip(e, g[scheme]):
        assert 0.75 * want <= got <= 1.25 * want, (scheme, got, want)
    assert abs(math.log2(e[0] / e[1]) - g["order_64_128"][scheme]) <= 0.1


# --- 5b. long runs on a static two-level mesh ----------------------------------------------

def _amr_advection(m, ic, params, T):
    """L1(rho) against the exact solution, area-weighted over the leaves, and the relative
    change of the total mass, after a run to time T."""
    U0 = w.evaluate_on_mesh(m, ic)
    o = Oracle(m, U0)
    run_to_time(o, params, T)
    U = o.get_state()
    area = np.array([np.prod(m.leaf_dx(b)[:2]) for b in range(m.nleaves)])[:, None, None, None]
    err = float((np.abs(U[:, 0] - w.evaluate_on_mesh(m, ic, t=T)[:, 0]) * area).sum() / (area.sum() * 256))
    mass0, mass1 = float((U0[:, 0] * area).sum()), float((U[:, 0] * area).sum())
    return err, (mass1 - mass0) / mass0, U


@pytest.mark.parametrize("scheme", SCHEMES)
def test_long_run_on_a_static_two_level_strip(scheme):
    """The 1D advection of Table 1 (Sec. 5) for one period (about 1000 and 2000 steps) with
    the middle half of the strip refined: the density wave crosses both coarse/fine
    interfaces, through the ghost fill of Sec. 4.3 and the reflux.  The mathematics fixes:
    the total mass to round-off (the update and the reflux are conservative); an error between
    those of the all-coarse and the all-fine meshes; second-order convergence when both levels
    are refined (order >= 1.7, the paper's uniform order here being 1.8-2.0); and the
    y-uniform solution staying y-uniform, bitwise, across levels.  A skipped reflux fails it;
    a ghost-fill mistake confined to the interface cells (a flipped prolongation slope,
    restriction by injection) moves the L1 error only at second order and is left to the
    ghost-fill pins above, which fail on either."""
    ic, strip = advection_1d, advection_strip
    params = P(gamma=1.4, c_cfl=0.8, scheme=scheme)

    e_coarse = _amr_advection(strip(64, False), ic, params, 1.0)[0]
    e_fine = _amr_advection(strip(128, False), ic, params, 1.0)[0]
    e64, dm64, U = _amr_advection(strip(64, True), ic, params, 1.0)
    e128, dm128, _ = _amr_advection(strip(128, True), ic, params, 1.0)
    assert 1.2 * e_fine < e64 < 0.8 * e_coarse, (e_fine, e64, e_coarse)
    assert math.log2(e64 / e128) >= 1.7, (e64, e128)
    assert abs(dm64) <= 1e-14 and abs(dm128) <= 1e-14, (dm64, dm128)
    assert np.all(U == U[:, :, :, :1, :]), "rows of a block differ"
    m = strip(64, True)
    fine = [b for b in range(m.nleaves) if m.leaves[b][1] == 1]
    for b in fine:                                    # the two fine rows of blocks agree
        twin = [c for c in fine if m.leaves[c][2] == m.leaves[b][2]]
        assert all(np.array_equal(U[b], U[c]) for c in twin)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_long_run_on_a_static_two_level_square(scheme):
    """The oblique 2D advection of Table 2 (Sec. 5) to t = 0.5 (about 600 and 1200 steps)
    with the central quarter of the domain refined, so that the wave crosses coarse/fine faces
    along both axes and their corners: total mass to round-off; an error between the
    all-coarse and all-fine meshes'; and refining both levels converges at the order of the
    uniform meshes (no worse by more than 0.1; at 32 and 64 cells per side the uniform order
    itself is only about 1.1-1.5)."""
    s3 = math.sqrt(3.0)
    params = P(gamma=1.4, scheme=scheme)

    def square(n, refined):
        return two_level_mesh(n, n // 16, (-0.5, -s3 / 2, 0), (0.5, s3 / 2, 1),
                              lambda i, j, nbx: refined and nbx // 4 <= i < 3 * nbx // 4
                              and nbx // 4 <= j < 3 * nbx // 4)

    u32 = _amr_advection(square(32, False), advection_2d, params, 0.5)[0]
    u64 = _amr_advection(square(64, False), advection_2d, params, 0.5)[0]
    a32, dm32, _ = _amr_advection(square(32, True), advection_2d, params, 0.5)
    a64, dm64, _ = _amr_advection(square(64, True), advection_2d, params, 0.5)
    assert u64 < a32 < u32, (u64, a32, u32)
    assert math.log2(a32 / a64) >= math.log2(u32 / u64) - 0.1, (a32, a64, u32, u64)
    assert abs(dm32) <= 1e-14 and abs(dm64) <= 1e-14, (dm32, dm64)


def _pulse(X, Y, Z, t=0.0, **_):
    """A narrow density pulse advected at unit speed on the periodic x in [-0.5, 0.5)."""
    xs = (X - t + 0.5) % 1.0 - 0.5
    rho = 1.0 + 0.5 * np.exp(-(xs / 0.06) ** 2)
    return conserved_from_primitive(rho, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1.0, 1.4)


def _pulse_run(scheme, nbx, max_level=0, every=4):
    """The pulse for one period on a strip of nbx blocks of 8^2 (one block high).  With
    max_level > 0 the refinement criterion (Sec. 4.5, on rho) settles the initial mesh and
    then runs every `every` steps, each regrid moving the state onto the new mesh (Sec. 4.3).
    Returns the final L1(rho) against the exact pulse (area-weighted, per 64-cell block), the
    largest relative change of the total mass, the number of distinct meshes and the final
    state and mesh."""
    m = w.uniform_mesh(2, 8, (nbx, 1), lo=(-0.5, 0, 0), hi=(0.5, 1.0 / nbx, 1))
    p = P(gamma=1.4, c_cfl=0.8, scheme=scheme)
    refine = dict(vars=("rho",), thr=0.05, coarsen=0.02, max_level=max_level)

    def area(mesh):
        return np.array([np.prod(mesh.leaf_dx(b)[:2]) for b in range(mesh.nleaves)])[:, None, None, None]

    def adapted(o, mesh):
        o.fill_ghosts()
        f, _ = o.flags(p, refine)
        new = w.Mesh(2, mesh.nb, mesh.problems, np.asarray(O.plan_regrid(mesh, f, max_level), dtype=np.int32))
        same = new.nleaves == mesh.nleaves and np.array_equal(new.leaves, mesh.leaves)
        return (o, mesh) if same else (o.regrid(new), new)

    o = Oracle(m, w.evaluate_on_mesh(m, _pulse))
    for _ in range(max_level + 1 if max_level else 0):      # settle on the initial condition
        o2, m2 = adapted(o, m)
        if m2 is m:
            break
        m = m2
        o = Oracle(m, w.evaluate_on_mesh(m, _pulse))
    mass0 = float((o.get_state()[:, 0] * area(m)).sum())
    drift, meshes, t, n = 0.0, {m.leaves.tobytes()}, 0.0, 0
    while t < 1.0 - 1e-14:
        if max_level and n > 0 and n % every == 0:
            o, m = adapted(o, m)
            meshes.add(m.leaves.tobytes())
            drift = max(drift, abs(float((o.get_state()[:, 0] * area(m)).sum()) - mass0) / mass0)
        o.fill_ghosts()
        dt = o.cfl(p)[0]
        if t + dt > 1.0:
            last = dict(p, dt_override=1.0 - t)
            o.cfl(last)
            o.step(last)
            t = 1.0
        else:
            o.step(p)
            t += dt
        n += 1
    U = o.get_state()
    drift = max(drift, abs(float((U[:, 0] * area(m)).sum()) - mass0) / mass0)
    A = area(m)
    err = float((np.abs(U[:, 0] - w.evaluate_on_mesh(m, _pulse, t=1.0)[:, 0]) * A).sum() / A.sum())
    return err, drift, len(meshes), U, m


@pytest.mark.parametrize("scheme", SCHEMES)
def test_long_run_that_regrids_as_it_goes(scheme):
    """A narrow density pulse crosses the periodic strip once (about 1400 steps) while the
    refinement criterion regrids every 4 steps, so the refined blocks travel with it (Sec. 4.5
    flags, the 2:1-balanced plan, Sec. 4.3 prolongation and restriction of the moved blocks).
    Fixed by the mathematics: the total mass holds to round-off through every step and regrid
    (the update, the reflux, the mean restriction and the minmod prolongation, whose slopes
    average to zero over the children, are all conservative); the strip stays y-uniform bitwise.
    And the run behaves as refinement should: the mesh changes dozens of times, and the final
    error is that of the mesh refined everywhere to within 25 %, against four times that on the
    coarse mesh.  A non-conservative regrid, a regrid that misplaces children, or flags that do
    not follow the pulse each fail it."""
    e_coarse = _pulse_run(scheme, 8)[0]                    # 64 cells
    e_fine = _pulse_run(scheme, 32)[0]                     # 256 cells, the finest level's spacing
    e, drift, nmesh, U, m = _pulse_run(scheme, 8, max_level=2)
    assert drift <= 1e-13, drift
    assert nmesh >= 20, nmesh
    assert e <= 1.25 * e_fine and e <= 0.25 * e_coarse, (e, e_fine, e_coarse)
    assert np.all(U == U[:, :, :, :1, :]), "rows of a block differ"


# --- 6. mirror and transpose symmetry ----------------------------------------------------

def _ens(X, Y, Z, **kw):
    U = ensemble_problem(X, Y, Z, seed=77)
    U[8] = 0.01 * np.sin(2 * math.pi * (2 * X + Y))   # nonzero psi too
    return U


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("op", ("mirror_x", "mirror_y", "transpose"))
def test_symmetry_2d(scheme, op):
    m = w.uniform_mesh(2, 16, (2, 2))
    U0 = w.evaluate_on_mesh(m, _ens)
    G0 = to_global(m, U0)

    def tf(G):
        G = G.copy()
        if op == "mirror_x":
            G = G[..., ::-1].copy(); G[[1, 4]] *= -1
        elif op == "mirror_y":
            G = G[:, :, ::-1, :].copy(); G[[2, 5]] *= -1
        else:
            G = np.swapaxes(G, 2, 3).copy(); G[[1, 2]] = G[[2, 1]]; G[[4, 5]] = G[[5, 4]]
        return G

    p = P(scheme=scheme, limiter="vanleer" if scheme == "lf" else "minmod", eta=1e-3)
    a = Oracle(m, U0)
    b = Oracle(m, from_global(m, tf(G0)))
    for _ in range(4):
        for o in (a, b):
            o.fill_ghosts()
        da, db = a.cfl(p), b.cfl(p)
        assert da[0] == db[0]
        a.step(p); b.step(p)
    A = tf(to_global(m, a.get_state()))
    B = to_global(m, b.get_state())
    for v in range(9):
        # psi is a small field born of cancellation: floor the scale at 1e-3
        scale = max(np.abs(B[v]).max(), 1e-3)
        assert np.abs(A[v] - B[v]).max() <= 1e-13 * scale, v


def test_symmetry_3d_lf():
    m = w.uniform_mesh(3, 8, (2, 2, 2))

    def ic(X, Y, Z, **_):
        rho = 1 + 0.1 * np.sin(2 * math.pi * (X + 2 * Y + 3 * Z))
        return conserved_from_primitive(rho, 0.1 * np.cos(2 * math.pi * Y), 0.05, -0.1 * np.sin(2 * math.pi * Z),
                                        0.3 + 0.05 * np.sin(2 * math.pi * Z), 0.2, 0.1 * np.cos(2 * math.pi * X),
                                        1.0, 5 / 3)
    U0 = w.evaluate_on_mesh(m, ic)
    G0 = to_global(m, U0)

    def tf(G):  # swap x and z
        G = np.swapaxes(G, 1, 3).copy()
        G[[1, 3]] = G[[3, 1]]; G[[4, 6]] = G[[6, 4]]
        return G

    p = P(scheme="lf", limiter="vanleer", eta=1e-3)
    a = Oracle(m, U0)
    b = Oracle(m, from_global(m, tf(G0)))
    for _ in range(2):
        for o in (a, b):
            o.fill_ghosts(); o.cfl(p); o.step(p)
    A = tf(to_global(m, a.get_state()))
    B = to_global(m, b.get_state())
    for v in range(9):
        assert np.abs(A[v] - B[v]).max() <= 1e-13 * max(np.abs(B[v]).max(), 1e-3), v


# --- 7. block-decomposition invariance ---------------------------------------------------

@pytest.mark.parametrize("scheme", SCHEMES)
def test_block_decomposition_invariance(scheme):
    p = P(scheme=scheme)
    res = []
    for nb, nbk in ((16, 4), (32, 2), (64, 1)):
        m = w.uniform_mesh(2, nb, (nbk, nbk))
        o = Oracle(m, w.evaluate_on_mesh(m, orszag_tang))
        for _ in range(3):
            o.fill_ghosts(); o.cfl(p); o.step(p)
        res.append(to_global(m, o.get_state()))
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])


def test_refined_everywhere_equals_uniform():
    p = P(scheme="lf", limiter="vanleer")
    m0 = w.uniform_mesh(2, 16, (4, 4))
    leaves = np.array([(0, 1, i, j, 0) for j in range(4) for i in range(4)], dtype=np.int32)
    m1 = w.Mesh(2, 16, [w.Problem((2, 2, 1))], leaves)
    outs = []
    for m in (m0, m1):
        o = Oracle(m, w.evaluate_on_mesh(m, orszag_tang))
        for _ in range(3):
            o.fill_ghosts(); o.cfl(p); o.step(p)
        outs.append(to_global(m0, o.get_state()) if m is m0 else None)
        if m is m1:
            U = o.get_state()
            G = np.zeros_like(outs[0])
            for b, (_, lv, i, j, k) in enumerate(m1.leaves):
                G[:, :, j * 16:(j + 1) * 16, i * 16:(i + 1) * 16] = U[b]
            outs[1] = G
    np.testing.assert_array_equal(outs[0], outs[1])


# --- 8. prolongation and restriction (Sec. 4.3) ------------------------------------------

def test_prolong_1d_cases():
    assert O.prolong_1d(1.0, 2.0, 1.0, True) == 2.0          # extremum: slope killed
    assert O.prolong_1d(1.0, 2.0, 1.0, False) == 2.0
    assert O.prolong_1d(0.0, 1.0, 3.0, True) == 1.25         # minmod(2, 1) = 1, +1/4
    assert O.prolong_1d(0.0, 1.0, 3.0, False) == 0.75
    assert O.prolong_1d(3.0, 1.0, 0.0, True) == 0.75         # minmod(-1, -2) = -1


def _linear(X, Y, Z, **_):
    out = np.empty((9,) + X.shape)
    for v in range(9):
        out[v] = 1.0 + 0.1 * v + (0.3 + 0.01 * v) * X - (0.2 - 0.02 * v) * Y + 0.05 * v * Z
    return out


@pytest.mark.parametrize("ndim", (2, 3))
def test_ghost_fill_linear_exact(ndim):
    """Same-level copy, restriction into coarse ghosts and minmod prolongation into fine
    ghosts all reproduce a linear field exactly (away from the outflow boundary)."""
    if ndim == 2:
        m = w.radial_amr_mesh(2, 8, (4, 4), 2, radii=(0.12, 0.3), bc=w.mesh.OUTFLOW)
    else:
        m = w.radial_amr_mesh(3, 4, (4, 4, 4), 1, radii=(0.2,), bc=w.mesh.OUTFLOW)
    o = Oracle(m, w.evaluate_on_mesh(m, _linear))
    assert o.fill_ghosts() == 0
    checked = 0
    for b in range(m.nleaves):
        G = o.get_ghosted(b)
        dx = m.leaf_dx(b)
        org = m.leaf_origin(b)
        n = m.nb + 4
        ii = np.arange(n)
        x = org[0] + (ii - 2 + 0.5) * dx[0]
        y = org[1] + (ii - 2 + 0.5) * dx[1]
        z = org[2] + (ii - 2 + 0.5) * dx[2] if ndim == 3 else np.array([0.0])
        Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
        want = _linear(Xg, Yg, Zg)
        coarse_dx = dx[0] * 2
        inside = (np.abs(Xg) < 0.5 - 3 * coarse_dx) & (np.abs(Yg) < 0.5 - 3 * coarse_dx)
        if ndim == 3:
            inside &= np.abs(Zg) < 0.5 - 3 * coarse_dx
        if not inside.any():
            continue
        diff = np.abs(G - want)[:, inside]
        checked += inside.sum()
        assert diff.max() <= 1e-13, (b, diff.max())
    assert checked > 0


def test_regrid_restrict_prolong_identity_and_conservation():
    m0 = w.uniform_mesh(2, 8, (2, 2))
    U0 = w.evaluate_on_mesh(m0, _ens)
    o0 = Oracle(m0, U0)
    o0.fill_ghosts()
    s0 = o0.conservation()
    leaves1 = np.array([(0, 1, 2 * i + a, 2 * j + b, 0) for j in range(2) for i in range(2)
                        for b in range(2) for a in range(2)], dtype=np.int32)
    m1 = w.Mesh(2, 8, m0.problems, leaves1)
    o1 = o0.regrid(m1)
    s1 = o1.conservation()
    np.testing.assert_allclose(s1, s0, rtol=1e-14, atol=1e-16)
    o1.fill_ghosts()
    o2 = o1.regrid(m0)
    np.testing.assert_allclose(o2.get_state(), U0, rtol=1e-14, atol=1e-15)


def test_unbalanced_mesh_rejected():
    # a level-2 leaf touching a level-0 leaf
    leaves = [(0, 0, 1, 0, 0), (0, 0, 0, 1, 0), (0, 0, 1, 1, 0)]
    leaves += [(0, 1, a, b, 0) for a in (0, 1) for b in (0, 1) if (a, b) != (1, 1)]
    leaves += [(0, 2, 2 + a, 2 + b, 0) for a in (0, 1) for b in (0, 1)]
    m = w.Mesh(2, 8, [w.Problem((2, 2, 1))], np.array(leaves, dtype=np.int32))
    with pytest.raises(ValueError):
        Oracle(m)


# --- 9. GLM cleaning reduces div B (Sec. 5, 2D divergence free test) --------------------

def _divb_l1(U, m):
    dx = m.leaf_dx(0)
    Bx = assemble_uniform(m, U, 4)[0]
    By = assemble_uniform(m, U, 5)[0]
    d = (np.roll(Bx, -1, 1) - np.roll(Bx, 1, 1)) / (2 * dx[0]) + (np.roll(By, -1, 0) - np.roll(By, 1, 0)) / (2 * dx[1])
    return np.abs(d).mean()


@pytest.mark.parametrize("scheme", ("lf", "weno"))
def test_glm_divb_reduction(scheme):
    """Field-loop advection (Sec. 5, 2D divergence free test): with GLM cleaning the mean
    |div B| stays at least an order of magnitude below the run without cleaning (c_h = 0),
    as the paper reports for its Fig. 10."""
    m = w.uniform_mesh(2, 16, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1))
    U0 = w.evaluate_on_mesh(m, field_loop)
    res = {}
    for mode in ("auto", "fixed"):
        o = Oracle(m, U0)
        run_to_time(o, P(scheme=scheme, limiter="minmod", ch_mode=mode, ch=0.0), 0.5)
        res[mode] = _divb_l1(o.get_state(), m)
    assert res["auto"] * 10 <= res["fixed"], res


# --- 10/11. WENO special cases and LF flux consistency -----------------------------------

def test_weno_special_cases():
    a, b = O.weno_faces(1.0, 2.0, 3.0)
    assert abs(a - 2.5) <= 1e-15 and abs(b - 1.5) <= 1e-15      # linear: exact
    a, b = O.weno_faces(4.0, 4.0, 4.0)
    assert a == 4.0 and b == 4.0                                 # constant: exact
    a, b = O.weno_faces(0.0, 0.0, 1.0)
    assert abs(a) < 1e-20                                        # discontinuity: smooth side
    # smooth data: second-order accurate face values
    errs = []
    for h in (0.0125, 0.00625, 0.003125):
        x0 = 0.3
        a, b = O.weno_faces(math.sin(x0 - h), math.sin(x0), math.sin(x0 + h))
        errs.append(abs(a - math.sin(x0 + h / 2)) + abs(b - math.sin(x0 - h / 2)))
    assert 1.8 <= math.log2(errs[1] / errs[2]) <= 2.2, errs


def test_limiters():
    assert O.limiter("minmod", 1.0, 2.0) == 1.0
    assert O.limiter("minmod", -1.0, -3.0) == -1.0
    assert O.limiter("minmod", -1.0, 3.0) == 0.0
    assert O.limiter("vanleer", 1.0, 3.0) == 1.5
    assert O.limiter("vanleer", 1.0, -3.0) == 0.0
    assert O.limiter("roe", 1.0, 2.0) == 1.0 and O.limiter("roe", 3.0, 2.0) == 2.0


def test_lf_flux_consistency_and_galilean_parts():
    wst = conserved_from_primitive(np.array(1.2), 0.3, -0.4, 0.2, 0.5, 0.7, -0.1, 0.9, 5 / 3, 0.05)
    for d in range(3):
        np.testing.assert_array_equal(O.lf_flux(d, wst, wst, 5 / 3, 1.3), O.flux(d, wst, 5 / 3, 1.3))
    # static state: the flux is the total pressure on the normal momentum only (+ GLM)
    st = conserved_from_primitive(np.array(1.0), 0, 0, 0, 0.6, 0.0, 0.0, 1.0, 5 / 3, 0.2)
    f = O.flux(0, st, 5 / 3, 2.0)
    np.testing.assert_allclose(f, [0, 1.0 + 0.18 - 0.36, 0, 0, 0.2, 0, 0, 0, 4.0 * 0.6], atol=1e-15)


# --- EGLM source terms (eqs. MHD-2, MHD-4) ------------------------------------------------

def test_eglm_momentum_source_cancels_divb_force():
    """B_x = 1 + 0.2 x (div B = 0.2): the flux gives dm_x/dt = B_x dB_x/dx; the EGLM source
    -(div B) B_x cancels it."""
    m = w.uniform_mesh(2, 16, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=w.mesh.OUTFLOW)

    def ic(X, Y, Z, **_):
        return conserved_from_primitive(np.ones_like(X), 0, 0, 0, 1 + 0.2 * X, 0, 0, 1.0, 5 / 3)

    U0 = w.evaluate_on_mesh(m, ic)
    dm = {}
    for eglm in (0, 1):
        o = Oracle(m, U0)
        p = P(scheme="lf", eglm=eglm, ch_mode="fixed", ch=0.0)
        o.fill_ghosts(); dt = o.cfl(p)[0]; o.step(p)
        G = assemble_uniform(m, o.get_state(), 1)[0]
        dm[eglm] = G[28:36, 28:36]
        X = assemble_uniform(m, U0, 4)[0][28:36, 28:36]
    np.testing.assert_allclose(dm[0], dt * X * 0.2, rtol=0.02)
    assert np.abs(dm[1]).max() < 0.02 * np.abs(dm[0]).max()


def test_eglm_energy_source():
    """psi = 0.3 x with B_x = 1, static: de/dt = -B . grad psi = -0.3 with EGLM, 0 without."""
    m = w.uniform_mesh(2, 16, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=w.mesh.OUTFLOW)

    def ic(X, Y, Z, **_):
        return conserved_from_primitive(np.ones_like(X), 0, 0, 0, 1.0, 0, 0, 1.0, 5 / 3, 0.3 * X)

    U0 = w.evaluate_on_mesh(m, ic)
    de = {}
    for eglm in (0, 1):
        o = Oracle(m, U0)
        p = P(scheme="mmc", eglm=eglm)
        o.fill_ghosts(); dt = o.cfl(p)[0]; o.step(p)
        de[eglm] = (assemble_uniform(m, o.get_state(), 7) - assemble_uniform(m, U0, 7))[0][28:36, 28:36]
    np.testing.assert_allclose(de[1], -0.3 * dt, rtol=0.02)
    assert np.abs(de[0]).max() < 0.02 * 0.3 * dt


# --- resistivity (Sec. 3.5) ---------------------------------------------------------------

def _res_strip(eta, n=64, T=0.5, eps=1e-3):
    m = w.uniform_mesh(2, 16, (n // 16, 1), lo=(0, 0, 0), hi=(1, 16.0 / n, 1))

    def ic(X, Y, Z, **_):
        return conserved_from_primitive(np.ones_like(X), 0, 0, 0, 0.0, eps * np.sin(2 * math.pi * X), 0, 1.0, 5 / 3)

    o = Oracle(m, w.evaluate_on_mesh(m, ic))
    run_to_time(o, P(scheme="lf", limiter="vanleer", eta=eta), T)
    return m, o.get_state()


def test_resistive_decay_rate():
    n, T, eta = 64, 0.5, 4e-3
    m, U1 = _res_strip(eta, n, T)
    _, U0 = _res_strip(0.0, n, T)
    by1 = assemble_uniform(m, U1, 5)[0, 0]
    by0 = assemble_uniform(m, U0, 5)[0, 0]
    x = (np.arange(n) + 0.5) / n
    s = np.sin(2 * math.pi * x)
    ratio = (by1 @ s) / (by0 @ s)
    h = 1.0 / n
    keff2 = (math.sin(2 * math.pi * h) / h) ** 2       # central difference of a central difference
    assert ratio == pytest.approx(math.exp(-eta * keff2 * T), rel=2e-3)


def test_resistive_terms_one_step_closed_form():
    """From a static state with B_y = eps sin(kx), one step with and without eta differs by
    exactly dt R (the resistive terms enter the final update only): dB_y = dt R_y and
    de = dt R_e, with the central-difference closed forms
      J_z = eps cos(kx) sin(kh)/h,  R_y = -eta eps (sin(kh)/h)^2 sin(kx),
      R_e = eta eps^2/2 (sin(kh)/h) (sin(2kh)/h) cos(2kx)   (Sec. 3.5)."""
    n, eta, eps = 64, 4e-3, 1e-2
    m = w.uniform_mesh(2, 16, (n // 16, 1), lo=(0, 0, 0), hi=(1, 16.0 / n, 1))

    def ic(X, Y, Z, **_):
        return conserved_from_primitive(np.ones_like(X), 0, 0, 0, 0.0, eps * np.sin(2 * math.pi * X), 0, 1.0, 5 / 3)

    U0 = w.evaluate_on_mesh(m, ic)
    out = {}
    for e in (0.0, eta):
        o = Oracle(m, U0)
        p = P(scheme="lf", limiter="vanleer", eta=e)
        o.fill_ghosts(); dt = o.cfl(p)[0]; o.step(p)
        out[e] = (dt, o.get_state())
    assert out[0.0][0] == out[eta][0]
    dt = out[eta][0]
    h, k = 1.0 / n, 2 * math.pi
    x = (np.arange(n) + 0.5) / n
    dby = assemble_uniform(m, out[eta][1], 5)[0, 0] - assemble_uniform(m, out[0.0][1], 5)[0, 0]
    de = assemble_uniform(m, out[eta][1], 7)[0, 0] - assemble_uniform(m, out[0.0][1], 7)[0, 0]
    sk = math.sin(k * h) / h
    np.testing.assert_allclose(dby, -dt * eta * eps * sk * sk * np.sin(k * x), rtol=1e-9, atol=1e-18)
    re = eta * eps * eps / 2 * sk * (math.sin(2 * k * h) / h) * np.cos(2 * k * x)
    np.testing.assert_allclose(de, dt * re, rtol=1e-6, atol=1e-20)


# --- 12. refinement estimator special cases (Sec. 4.5) -----------------------------------

def _flags_for(ic, refine, nbk=2, level_leaves=None):
    m = w.uniform_mesh(2, 8, (nbk, nbk), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=w.mesh.OUTFLOW)
    o = Oracle(m, w.evaluate_on_mesh(m, ic))
    o.fill_ghosts()
    return o.flags(P(), refine)


def test_estimator_constant_and_linear():
    f, est = _flags_for(uniform_state, dict(vars=("rho", "p"), thr=0.2, coarsen=0.1, max_level=3))
    assert np.all(est == 0.0) and np.all(f == 0)  # level 0 cannot coarsen

    g = 0.5

    def lin(X, Y, Z, **_):
        return conserved_from_primitive(2.0 + g * X, 0, 0, 0, 0, 0, 0, 1.0, 5 / 3)
    f, est = _flags_for(lin, dict(vars=("rho",), thr=0.2, max_level=3), nbk=4)
    # linear rho: |du| = sqrt(3)/2 |2 g h| and |d2u| = 0 at every cell whose neighbours are
    # linear too, i.e. in blocks away from the outflow boundary; the block maximum sits at
    # the smallest rho, the first ghost ring cell at x = block_lo - h/2
    h = 1.0 / 32
    m = w.uniform_mesh(2, 8, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1))
    for b, (_, lv, i, j, k) in enumerate(m.leaves):
        if i in (1, 2) and j in (1, 2):
            xlo = -0.5 + i * 8 * h
            want = 0.6 * (math.sqrt(3) / 2) * (2 * g * h) / (2.0 + g * (xlo - h / 2) + 1e-12)
            assert est[b] == pytest.approx(want, rel=1e-12)


def test_estimator_second_difference_term():
    """rho = a + b x^2 + c y^2 has the same nonzero second difference at every cell, so the
    (1-B)|d2u| / (|du| + F(|u|+eps)) term is pinned against its closed form: a dropped (1-B),
    eps outside the F factor (eps is 0.3 here, comparable to |u|), or |d2x| + |d2y| in place
    of sqrt(d2x^2 + d2y^2) each move the block maxima by far more than the tolerance."""
    a, b, c, eps = 0.2, 40.0, 20.0, 0.3
    refine = dict(vars=("rho",), thr=0.36, coarsen=0.1, max_level=3, bias=0.6, filter=0.05,
                  eps_rho=eps)

    def quad(X, Y, Z, **_):
        return conserved_from_primitive(a + b * X * X + c * Y * Y, 0, 0, 0, 0, 0, 0, 1.0, 5 / 3)

    m = w.uniform_mesh(2, 8, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1), bc=w.mesh.OUTFLOW)
    o = Oracle(m, w.evaluate_on_mesh(m, quad))
    o.fill_ghosts()
    f, est = o.flags(P(), refine)
    h = 1.0 / 32
    # the estimator runs over the interior and the first ghost ring; in the inner blocks
    # (away from the outflow boundary) every cell there and its neighbours hold the quadratic
    k = np.arange(-1, 9) + 0.5
    checked = 0
    for blk, (_, lv, i, j, _k) in enumerate(m.leaves):
        if i not in (1, 2) or j not in (1, 2):
            continue
        X, Y = np.meshgrid(-0.5 + (i * 8 + k) * h, -0.5 + (j * 8 + k) * h)
        first, full = quadratic_estimate(a, b, c, h, eps, refine, X, Y)
        assert est[blk] == pytest.approx(float(full.max()), rel=1e-9)
        # the flag decision rests on the second-difference term: the first-difference term
        # alone stays below the threshold, the whole estimator exceeds it
        assert float(first.max()) < 0.9 * refine["thr"] < 1.1 * refine["thr"] < float(full.max())
        assert f[blk] == 1
        checked += 1
    assert checked == 4


def test_estimator_second_difference_mutations_detected():
    """The closed form above separates the plausible misreadings of the Sec. 4.5 estimator by
    more than the tolerance used there (so each would fail that test)."""
    a, b, c, eps, h = 0.2, 40.0, 20.0, 0.3, 1.0 / 32
    r = dict(bias=0.6, filter=0.05)
    k = np.arange(-1, 9) + 0.5
    X, Y = np.meshgrid(-0.5 + (8 + k) * h, -0.5 + (8 + k) * h)
    first, full = quadratic_estimate(a, b, c, h, eps, r, X, Y)
    u = a + b * X * X + c * Y * Y
    du = math.sqrt(3.0) / 2.0 * 4.0 * h * np.sqrt(b * b * X * X + c * c * Y * Y)
    d2 = 2.0 * h * h * math.sqrt(b * b + c * c)
    d2_abs = 2.0 * h * h * (abs(b) + abs(c))
    variants = {
        "no (1-B)": first + d2 / (du + r["filter"] * (u + eps)),
        "eps outside F": first + (1 - r["bias"]) * d2 / (du + r["filter"] * u + eps),
        "|d2x|+|d2y|": first + (1 - r["bias"]) * d2_abs / (du + r["filter"] * (u + eps)),
        "no sqrt(3)/2 in the denominator": first + (1 - r["bias"]) * d2 / (du / (math.sqrt(3) / 2)
                                                                           + r["filter"] * (u + eps)),
    }
    for name, v in variants.items():
        assert abs(float(v.max()) / float(full.max()) - 1.0) > 1e-3, name


def test_estimator_flags_refine_and_coarsen():
    def jump(X, Y, Z, **_):
        return conserved_from_primitive(np.where(X > 0.3, 2.0, 1.0), 0, 0, 0, 0, 0, 0, 1.0, 5 / 3)
    f, est = _flags_for(jump, dict(vars=("rho",), thr=0.2, coarsen=0.1, max_level=3), nbk=4)
    m = w.uniform_mesh(2, 8, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1))
    for b, (_, lv, i, j, k) in enumerate(m.leaves):
        if i == 3:   # x in [0.25, 0.5]: the only blocks whose cells see the jump at 0.3
            assert f[b] == 1
        else:
            assert f[b] == 0 and est[b] == 0.0


# --- Brio-Wu shock tube: robustness and exact 1D symmetry (Sec. 5) -----------------------

@pytest.mark.parametrize("scheme", ("lf", "weno"))
def test_brio_wu_robust_and_one_dimensional(scheme):
    n = 256
    m = w.uniform_mesh(2, 16, (n // 16, 1), lo=(-0.5, 0, 0), hi=(0.5, 16.0 / n, 1),
                       bc=((w.mesh.OUTFLOW, w.mesh.OUTFLOW), (0, 0), (0, 0)))
    o = Oracle(m, w.evaluate_on_mesh(m, brio_wu))
    run_to_time(o, P(gamma=2.0, scheme=scheme, limiter="minmod"), 0.1)
    U = o.get_state()
    assert np.isfinite(U).all() and (U[:, 0] > 0).all()
    # every row identical (the y direction is exactly uniform)
    G = np.stack([assemble_uniform(m, U, v)[0] for v in range(9)])
    assert np.all(G == G[:, :1, :])
    rho = G[0, 0]
    assert rho[:n // 4].mean() > 0.9 and rho[-n // 4:].mean() < 0.2


# --- MMC reduces to Lax-Wendroff for a linear wave of constant speed (Sec. 3.1) ---------

@pytest.mark.parametrize("sign", (1, -1))
@pytest.mark.parametrize("mode", (1, 3, 7))
def test_mmc_unlimited_is_lax_wendroff_on_the_glm_pair(sign, mode):
    """The (B_x, psi) pair of the x sweep is linear with the fixed speed c_h (Q4), so on a
    y-uniform strip with rho, v, p, B_y, B_z uniform the characteristic variable
    w = psi + sign c_h B_x is advected at sign c_h and nothing else feeds back into it.
    MMC with phi = 1 then reduces by hand to the Lax-Wendroff scheme: h = c_h w_i is the
    upwind flux, u~ the upwind predictor, g+ = c_h (w~_{i+1} - w_i), so
    fhat = c_h (w_i + (1 - nu)(w_{i+1} - w_i) / 2), whose one-step factor on
    exp(i theta j) is 1 - i nu sin(theta) - nu^2 (1 - cos(theta)) (nu = sign c_h dt / dx).
    A dropped 1/2, a g term on the wrong face or a predictor with the wrong sign each
    change that factor."""
    n, nb, ch = 64, 16, 2.0
    m = w.uniform_mesh(2, nb, (n // nb, 1), lo=(0, 0, 0), hi=(1, nb / n, 1))
    dx = 1.0 / n
    nu = 0.4
    dt = nu * dx / ch
    A, phi0 = 1e-2, 0.3
    theta = 2 * math.pi * mode / n

    def ic(X, Y, Z, **_):
        wv = A * np.cos(2 * math.pi * mode * (X - dx / 2) + phi0)      # theta j + phi0
        U = conserved_from_primitive(np.ones_like(X), 0.0, 0.0, 0.0, wv / (2 * sign * ch), 0.0, 0.0,
                                     1.0, 5 / 3)
        U[8] = wv / 2
        return U
    U0 = w.evaluate_on_mesh(m, ic)
    o = Oracle(m, U0)
    p = P(scheme="mmc", limiter="none", eglm=0, ch_mode="fixed", ch=ch, cp_mode="fixed", cp=0.0,
          dt_override=dt)
    o.fill_ghosts()
    o.cfl(p)
    o.step(p)
    U = o.get_state()
    wnew = assemble_uniform(m, U, 8)[0, 0] + sign * ch * assemble_uniform(m, U, 4)[0, 0]
    wother = assemble_uniform(m, U, 8)[0, 0] - sign * ch * assemble_uniform(m, U, 4)[0, 0]
    j = np.arange(n)
    G = 1 - 1j * (sign * nu) * math.sin(theta) - nu * nu * (1 - math.cos(theta))
    want = np.real(G * A * np.exp(1j * (theta * j + phi0)))
    np.testing.assert_allclose(wnew, want, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wother, 0.0, rtol=0, atol=1e-15)


# --- MMC with a varying speed: phi = 0 is Rusanov, phi = 1 a closed four-flux form --------

def _np_flux(d, U, gamma, ch):
    """EGLM-MHD flux along d (eqs. MHD-1 to MHD-5 without their sources), written out here
    from the equations on global arrays U[9, nz, ny, nx], independently of the oracle."""
    rho, m, B, e, psi = U[0], U[1:4], U[4:7], U[7], U[8]
    v = m / rho
    b2 = (B * B).sum(axis=0)
    p = (gamma - 1.0) * (e - 0.5 * (m * v).sum(axis=0) - 0.5 * b2)
    pt = p + 0.5 * b2
    F = np.empty_like(U)
    F[0] = m[d]
    for j in range(3):
        F[1 + j] = m[j] * v[d] - B[j] * B[d] + (pt if j == d else 0.0)
        F[4 + j] = psi if j == d else v[d] * B[j] - v[j] * B[d]
    F[7] = (e + pt) * v[d] - B[d] * (B * v).sum(axis=0)
    F[8] = ch * ch * B[d]
    return F


def _np_speed(d, U, gamma):
    """|v_d| plus the fast magnetosonic speed along d (reading Q2), from its closed form."""
    rho, m, B, e = U[0], U[1:4], U[4:7], U[7]
    b2 = (B * B).sum(axis=0)
    p = np.maximum((gamma - 1.0) * (e - 0.5 * (m * m).sum(axis=0) / rho - 0.5 * b2), 0.0)
    a2, va2, vd2 = gamma * p / rho, b2 / rho, B[d] ** 2 / rho
    s = a2 + va2
    cf = np.sqrt(0.5 * (s + np.sqrt(np.maximum(s * s - 4.0 * a2 * vd2, 0.0))))
    return np.abs(m[d] / rho) + cf


def _nxt(A, d):
    return np.roll(A, -1, axis=A.ndim - 1 - d)        # value at i+1 along d (periodic)


def _prv(A, d):
    return np.roll(A, 1, axis=A.ndim - 1 - d)


def _per_component(d, a, ch):
    """A face speed for every component: c_h for the (B_d, psi) pair (Q4), else a."""
    A = np.broadcast_to(a, (9,) + a.shape).copy()
    A[4 + d] = ch
    A[8] = ch
    return A


def _varying_state(X, Y, Z, gamma=5.0 / 3.0, ndim=2, **_):
    """A smooth periodic state in which every variable, and so the signal speed along every
    axis, varies in every direction."""
    t = 2.0 * math.pi
    Z = Z * (1.0 if ndim == 3 else 0.0)
    rho = 1.0 + 0.3 * np.sin(t * X) * np.cos(t * Y) + 0.15 * np.cos(t * (Z + X))
    vx = 0.2 + 0.4 * np.sin(t * (Y + Z))
    vy = -0.1 + 0.3 * np.sin(t * (X - Z) + 0.4)
    vz = 0.25 * np.cos(t * (X + Y))
    bx = 0.7 + 0.2 * np.cos(t * Y)
    by = 0.4 * np.sin(t * (X + Z) + 1.0)
    bz = 0.3 * np.cos(t * (X - Y))
    p = 0.6 + 0.25 * np.cos(t * (X + 2.0 * Y + Z))
    psi = 0.05 * np.sin(t * (X + Y + Z))
    return conserved_from_primitive(rho, vx, vy, vz, bx, by, bz, p, gamma, psi)


def _mmc_one_step(ndim, limiter, ch, dt):
    nb = 16 if ndim == 2 else 8
    m = w.uniform_mesh(ndim, nb, (2, 2, 2))
    U0 = w.evaluate_on_mesh(m, _varying_state, ndim=ndim)
    o = Oracle(m, U0)
    p = P(scheme="mmc", limiter=limiter, eglm=0, ch_mode="fixed", ch=ch, cp_mode="fixed", cp=0.0,
          dt_override=dt)
    o.fill_ghosts()
    o.cfl(p)
    assert o.step(p) == 0
    return to_global(m, U0), to_global(m, o.get_state()), 1.0 / (2 * nb)


def _update(U, F, lam):
    return U - sum(lam * (F[d] - _prv(F[d], d)) for d in range(len(F)))


@pytest.mark.parametrize("ndim", (2, 3))
def test_mmc_first_order_part_is_rusanov(ndim):
    """MMC's flux is h plus limited g terms (Sec. 3.1); with phi = 0 (an oracle test option)
    only h = f+_i + f-_{i+1} remains, and with f+- = (f +- alpha u)/2 sharing the face's speed
    that is, by hand, the Rusanov (local Lax-Friedrichs) flux
    (f(u_i) + f(u_{i+1}))/2 - alpha (u_{i+1} - u_i)/2.  On a state whose speed varies along
    every axis, the step equals that textbook scheme with alpha = max(alpha_d(u_i),
    alpha_d(u_{i+1})) per face and axis (c_h for the (B_d, psi) pair): the speeds of h are the
    face's two cells.  Per-cell speeds, or the maximum over the face's four-cell stencil,
    move the result by orders of magnitude more than the tolerance (checked here)."""
    gamma, ch = 5.0 / 3.0, 2.5
    dt = 2e-3
    U, got, dx = _mmc_one_step(ndim, "zero", ch, dt)
    lam = dt / dx

    def rusanov(speed):
        F = []
        for d in range(ndim):
            Ur = _nxt(U, d)
            A = _per_component(d, speed(d, U, Ur), ch)
            F.append(0.5 * (_np_flux(d, U, gamma, ch) + _np_flux(d, Ur, gamma, ch)) - 0.5 * A * (Ur - U))
        return _update(U, F, lam)

    face = lambda d, Ul, Ur: np.maximum(_np_speed(d, Ul, gamma), _np_speed(d, Ur, gamma))
    want = rusanov(face)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    # the readings this excludes
    stencil = lambda d, Ul, Ur: np.maximum(face(d, _prv(Ul, d), Ul), face(d, Ur, _nxt(Ur, d)))
    assert np.abs(rusanov(stencil) - got).max() > 1e-6
    per_cell = [rusanov(lambda d, Ul, Ur: _np_speed(d, Ul, gamma)), rusanov(lambda d, Ul, Ur: _np_speed(d, Ur, gamma))]
    assert min(np.abs(r - got).max() for r in per_cell) > 1e-6


@pytest.mark.parametrize("ndim", (2, 3))
def test_mmc_unlimited_flux_closed_form_with_varying_speed(ndim):
    """With phi = 1 (Sec. 3.1, an oracle test option) the MMC face flux h + (g+ - g-)/2, with
    g+_{i+1/2} = f~+_{i+1} - f+_i and g-_{i+1/2} = f-_{i+1} - f~-_i, collapses by hand to
    (f_i + f_{i+1} + f~_i + f~_{i+1})/4 - alpha (u_{i+1} - u_i)/4 + alpha~ (u~_{i+1} - u~_i)/4,
    u~ the Rusanov predictor of the whole (unsplit) step.  On a state whose speed varies
    along every axis, the step equals that form with alpha from u_i, u_{i+1} and alpha~ from
    u~_i, u~_{i+1} (reading Q3'): alpha~ taken from u, alpha~ = alpha, or a predictor over
    half the step each miss it by far more than the tolerance (checked here)."""
    gamma, ch = 5.0 / 3.0, 2.5
    dt = 2e-3
    U, got, dx = _mmc_one_step(ndim, "none", ch, dt)
    lam = dt / dx

    def face(d, Ul, Ur):
        return np.maximum(_np_speed(d, Ul, gamma), _np_speed(d, Ur, gamma))

    def step(pred_dt, tilde_speed_from_u=False, tilde_speed_is_alpha=False):
        H = []
        for d in range(ndim):
            Ur = _nxt(U, d)
            A = _per_component(d, face(d, U, Ur), ch)
            H.append(0.5 * (_np_flux(d, U, gamma, ch) + _np_flux(d, Ur, gamma, ch)) - 0.5 * A * (Ur - U))
        Ut = _update(U, H, pred_dt / dx)
        F = []
        for d in range(ndim):
            Ur, Utr = _nxt(U, d), _nxt(Ut, d)
            A = _per_component(d, face(d, U, Ur), ch)
            if tilde_speed_is_alpha:
                At = A
            else:
                At = _per_component(d, face(d, U, Ur) if tilde_speed_from_u else face(d, Ut, Utr), ch)
            F.append(0.25 * (_np_flux(d, U, gamma, ch) + _np_flux(d, Ur, gamma, ch) + _np_flux(d, Ut, gamma, ch)
                             + _np_flux(d, Utr, gamma, ch)) - 0.25 * A * (Ur - U) + 0.25 * At * (Utr - Ut))
        return _update(U, F, lam)

    want = step(dt)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    for wrong in (step(dt, tilde_speed_from_u=True), step(dt, tilde_speed_is_alpha=True), step(dt / 2)):
        assert np.abs(wrong - got).max() > 1e-8


def _sweby_phi(kind, th):
    if kind == "minmod":
        return np.maximum(0.0, np.minimum(1.0, th))
    if kind == "vanleer":
        return (th + np.abs(th)) / (1.0 + np.abs(th))
    return np.where(np.abs(th) <= 1.0, th, 1.0)       # Sec. 3.1's phi(r)


@pytest.mark.parametrize("limiter", ("minmod", "vanleer", "roe"))
@pytest.mark.parametrize("sign", (1, -1))
def test_mmc_limited_is_sweby_flux_limited_lax_wendroff_on_the_glm_pair(limiter, sign):
    """With a constant speed MMC's limited flux is, by hand, Sweby's flux-limited
    Lax-Wendroff flux (LeVeque, Finite Volume Methods, Sec. 6.12): on the (B_x, psi) pair,
    linear with the fixed speed c_h (Q4), the characteristic variable w = psi + sign c_h B_x
    is advected at sign c_h, h is the upwind flux, g = c_h (1 - nu)(w_{i+1} - w_i) on the
    upwind side and zero on the other, and r is the ratio of the upwind neighbour's jump to
    the face's, so fhat = c w_up + c (1 - nu) phi(theta)(w_{i+1} - w_i)/2.  A ratio taken
    from the wrong neighbour, a g with the wrong sign, or phi(r) applied as phi(1/r) fails
    it on this profile with extrema, jumps and a plateau."""
    n, nb, ch = 64, 16, 2.0
    m = w.uniform_mesh(2, nb, (n // nb, 1), lo=(0, 0, 0), hi=(1, nb / n, 1))
    dx = 1.0 / n
    nu = 0.4
    dt = nu * dx / ch
    A = 1e-2

    def profile(j):
        return A * (np.cos(2 * math.pi * 3 * j / n + 0.3) + 0.8 * ((j >= 20) & (j < 34)) - 0.5 * ((j >= 44) & (j < 52)))

    def ic(X, Y, Z, **_):
        j = np.rint(X / dx - 0.5)
        wv = profile(j)
        U = conserved_from_primitive(np.ones_like(X), 0.0, 0.0, 0.0, wv / (2 * sign * ch), 0.0, 0.0, 1.0, 5 / 3)
        U[8] = wv / 2
        return U

    o = Oracle(m, w.evaluate_on_mesh(m, ic))
    p = P(scheme="mmc", limiter=limiter, eglm=0, ch_mode="fixed", ch=ch, cp_mode="fixed", cp=0.0,
          dt_override=dt)
    o.fill_ghosts()
    o.cfl(p)
    assert o.step(p) == 0
    U = o.get_state()
    got = assemble_uniform(m, U, 8)[0, 0] + sign * ch * assemble_uniform(m, U, 4)[0, 0]
    other = assemble_uniform(m, U, 8)[0, 0] - sign * ch * assemble_uniform(m, U, 4)[0, 0]

    w0 = profile(np.arange(n).astype(float))
    jump = np.roll(w0, -1) - w0                                   # w_{i+1} - w_i at face i+1/2
    up = np.roll(jump, 1) if sign > 0 else np.roll(jump, -1)      # the upwind neighbour's jump
    safe = np.where(jump == 0.0, 1.0, jump)
    lim = np.where(jump == 0.0, 0.0, _sweby_phi(limiter, up / safe) * jump)
    F = (ch * w0 if sign > 0 else -ch * np.roll(w0, -1)) + 0.5 * ch * (1 - nu) * lim
    want = w0 - dt / dx * (F - np.roll(F, 1))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(other, 0.0, rtol=0, atol=1e-15)
    assert np.abs(lim).max() > 0 and np.count_nonzero(lim != jump) > 4   # the limiter acts


# --- domain of dependence: the face speeds are local ---------------------------------------

@pytest.mark.parametrize("scheme,limiter", [("mmc", "minmod"), ("mmc", "vanleer"), ("lf", "vanleer"),
                                            ("weno", "minmod")])
@pytest.mark.parametrize("at", [(7, 9), (15, 16), (0, 31)])
def test_one_step_domain_of_dependence(scheme, limiter, at):
    """One step with dt, c_h and c_p fixed: raising the pressure of one cell, so that its
    signal speed becomes the largest in the domain, changes the new state only within two
    cells of it (Chebyshev distance, across block edges and the periodic wrap) and leaves every
    other cell bitwise as it was.  Two ghost layers bound every stencil of the schemes (Sec.
    3.1-3.3, 3.7), and the MMC speeds taken from the relevant range of u and u~ (Sec. 3.1) are
    pinned to a local range: a global speed, or one gathered farther out, would move cells
    beyond it.  For WENO-RK2 the bound is twice two cells (two stages)."""
    m = w.uniform_mesh(2, 16, (2, 2))                     # 32 x 32, periodic
    U0 = w.evaluate_on_mesh(m, orszag_tang)
    p = P(scheme=scheme, limiter=limiter, dt_override=2e-3, ch_mode="fixed", ch=1.5, cp_mode="fixed", cp=0.5)

    def one_step(U):
        o = Oracle(m, U)
        o.fill_ghosts()
        o.cfl(p)
        assert o.step(p) == 0
        return to_global(m, o.get_state())

    U1 = U0.copy()
    gi, gj = at
    bl = [k for k in range(m.nleaves) if tuple(m.leaves[k][2:4]) == (gi // 16, gj // 16)][0]
    U1[bl, 7, 0, gj % 16, gi % 16] += 4.0                 # e: p about 27x, the largest speed
    A, B = one_step(U0), one_step(U1)
    moved = np.abs(A - B).max(axis=0)[0]                  # [y][x]
    n = 32
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    dxp = np.minimum(np.abs(x - gi), n - np.abs(x - gi))
    dyp = np.minimum(np.abs(y - gj), n - np.abs(y - gj))
    reach = 4 if scheme == "weno" else 2
    far = np.maximum(dxp, dyp) > reach
    assert np.all(moved[far] == 0.0), np.argwhere(far & (moved != 0.0))[:5]
    assert moved[gj, gi] > 0.0
    assert np.count_nonzero(moved[~far]) > 5
