"""Oracle pins for the HLLD interface flux of LF and WENO (Sec. 3.2, Sec. 5 Brio-Wu).

The paper names HLLD (Miyoshi & Kusano 2005) among MAP's approximate Riemann solvers and
compares it with HLLC on the Brio-Wu tube without printing it; the oracle restates the
published solver.  Pinned against what the mathematics fixes:
* with B = 0 and psi = 0 it is the textbook HLLC of the Euler equations (Toro's star state
  with Davis speed bounds), written out independently in the HLLC pins;
* it is consistent (F(U, U) = F(U));
* it is exact for an isolated contact, with or without a normal field;
* it is exact for an isolated rotational (Alfven) discontinuity at rest, of either family,
  which HLLC and f_m smear: such a discontinuity stays put under LF and WENO;
* the 2D mirror and transpose symmetries hold;
* on the Brio-Wu shock tube it stays positive and lies closer to a fine-grid solution than
  HLLC (the paper's comparison of Fig. 7);
* with reflux it conserves on AMR like every flux-form update.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as w
from oracle import Oracle
from oracle import oracle as O
from tests.helpers import assemble_uniform
from tests.test_hllc_pins import G53, _brio_wu, _cons, _euler_hllc, _rand_state


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_is_euler_hllc_without_field(d):
    rng = np.random.default_rng(140 + d)
    for trial in range(200):
        a, b = _rand_state(rng, False, False), _rand_state(rng, False, False)
        if trial % 10 == 0:                     # supersonic to either side
            sgn = 3.0 if trial % 20 == 0 else -3.0
            va, vb = a[1:4] / a[0], b[1:4] / b[0]
            va[d] += sgn
            vb[d] += sgn
            a = _cons(a[0], va, np.zeros(3), 1.0)
            b = _cons(b[0], vb, np.zeros(3), 0.5)
        got = O.hlld_flux(d, a, b, G53, 1.0)
        ref = _euler_hllc(d, a, b, G53)
        idx = [0, 1, 2, 3, 7]
        np.testing.assert_allclose(got[idx], ref[idx], rtol=1e-12, atol=1e-13)
        assert got[4 + d] == 0.0 and got[8] == 0.0


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_consistent_with_the_physical_flux(d):
    rng = np.random.default_rng(17 + d)
    for _ in range(100):
        U = _rand_state(rng)
        ch = rng.uniform(0.5, 3.0)
        np.testing.assert_allclose(O.hlld_flux(d, U, U, G53, ch), O.flux(d, U, G53, ch), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("u0", [-0.4, 0.0, 0.3])
@pytest.mark.parametrize("bn", [0.0, 0.7])
def test_hlld_exact_for_an_isolated_contact(d, u0, bn):
    """Only the density jumps: the exact interface flux is that of the upwind state."""
    v = np.zeros(3); v[d] = u0; v[(d + 1) % 3] = 0.2; v[(d + 2) % 3] = -0.1
    B = np.zeros(3); B[d] = bn; B[(d + 1) % 3] = 0.5; B[(d + 2) % 3] = -0.3
    a = _cons(1.0, v, B, 0.8)
    b = _cons(0.25, v, B, 0.8)
    ch = 2.0
    up = a if u0 >= 0 else b
    np.testing.assert_allclose(O.hlld_flux(d, a, b, G53, ch), O.flux(d, up, G53, ch), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hlld_carries_the_tangential_field_with_the_mass_when_bn_is_zero(d):
    """With no normal field the tangential field is frozen into the fluid: B_t / rho is carried
    with the mass.  HLLD's outer star states scale B_t with the density, so in every region of
    its fan the induction flux is (B_t / rho of the side upwind of the contact) times the mass
    flux, to round-off; the HLLC here (HLL-state field) does not do so."""
    rng = np.random.default_rng(91 + d)
    hllc_off = 0.0
    for trial in range(200):
        a, b = _rand_state(rng, True, False), _rand_state(rng, True, False)
        for U in (a, b):
            U[7] -= 0.5 * U[4 + d] ** 2                    # remove B_d at unchanged pressure
            U[4 + d] = 0.0
        f = O.hlld_flux(d, a, b, G53, 1.0)
        # the side upwind of the contact: the mass flux's direction fixes it where it is nonzero
        up = a if f[0] > 0 else b
        t = [j for j in range(3) if j != d]
        for j in t:
            np.testing.assert_allclose(f[4 + j], up[4 + j] / up[0] * f[0], rtol=1e-11, atol=1e-13)
        g = O.hllc_flux(d, a, b, G53, 1.0)
        hllc_off = max(hllc_off, max(abs(g[4 + j] - (a if g[0] > 0 else b)[4 + j] / (a if g[0] > 0 else b)[0] * g[0])
                                     for j in t))
    assert hllc_off > 1e-2


def _rotational(d, rho, bn, s, bt, c, p=1.0, gamma=G53):
    """A state on one side of a rotational discontinuity at rest along d: normal velocity
    u = s B_n / sqrt(rho) (the discontinuity moves at u - s B_n / sqrt(rho) = 0), tangential
    velocity c + s B_t / sqrt(rho).  The conservation laws across the jump then hold for any
    rotation of B_t at fixed |B_t| (rho, p, u and B_n continuous)."""
    t = [j for j in range(3) if j != d]
    v = np.zeros(3)
    B = np.zeros(3)
    v[d] = s * bn / math.sqrt(rho)
    B[d] = bn
    for q in range(2):
        B[t[q]] = bt[q]
        v[t[q]] = c[q] + s * bt[q] / math.sqrt(rho)
    return _cons(rho, v, B, p, gamma=gamma)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("s", [1, -1])
@pytest.mark.parametrize("bn", [0.8, -0.6])
def test_hlld_exact_for_a_rotational_discontinuity_at_rest(d, s, bn):
    """The Alfven waves are HLLD's inner waves: for an isolated rotational discontinuity at
    rest the flux is F(U_L) = F(U_R) to round-off; HLLC, which has no Alfven wave, and f_m
    are off by O(1)."""
    rho, ch = 1.7, 2.5
    c = (0.2, -0.15)
    th = 1.1
    a = _rotational(d, rho, bn, s, (0.9, 0.3), c)
    b = _rotational(d, rho, bn, s, (0.9 * math.cos(th) - 0.3 * math.sin(th), 0.9 * math.sin(th) + 0.3 * math.cos(th)), c)
    Fa, Fb = O.flux(d, a, G53, ch), O.flux(d, b, G53, ch)
    np.testing.assert_allclose(Fa, Fb, rtol=0, atol=1e-14)              # the jump conditions hold
    np.testing.assert_allclose(O.hlld_flux(d, a, b, G53, ch), Fa, rtol=0, atol=1e-13)
    assert np.abs(O.hllc_flux(d, a, b, G53, ch) - Fa).max() > 1e-2
    assert np.abs(O.lf_flux(d, a, b, G53, ch) - Fa).max() > 1e-2


@pytest.mark.parametrize("scheme", ["lf", "weno"])
def test_rotational_discontinuity_at_rest_stays_put(scheme):
    """A strip of two states joined by rotational discontinuities at rest (x = 0 and the
    periodic wrap): ten steps of LF (minmod) or WENO with HLLD change no cell by more than
    round-off; with HLLC both jumps smear."""
    m = w.uniform_mesh(2, 8, (8, 1), lo=(-0.5, 0, 0), hi=(0.5, 0.125, 1))
    bn, rho, s = 0.8, 1.7, -1
    c = (0.2, -0.15)
    a = _rotational(0, rho, bn, s, (0.9, 0.3), c)
    b = _rotational(0, rho, bn, s, (-0.3, 0.9), c)

    def ic(X, Y, Z, **_):
        left = (X < 0.0)[None]
        return np.where(left, a.reshape(9, 1, 1, 1), b.reshape(9, 1, 1, 1)) + 0.0 * X

    U0 = w.evaluate_on_mesh(m, ic)
    moved = {}
    for rs in ("hlld", "hllc"):
        o = Oracle(m, U0)
        o.advance(dict(scheme=scheme, riemann=rs, limiter="minmod"), 10)
        moved[rs] = np.abs(o.get_state() - U0).max()
    assert moved["hlld"] <= 1e-12, moved
    assert moved["hllc"] > 1e-3, moved


def _ens(X, Y, Z, **kw):
    U = w.problems.ensemble_problem(X, Y, Z, seed=77)
    U[8] = 0.01 * np.sin(2 * math.pi * (2 * X + Y))
    return U


@pytest.mark.parametrize("scheme", ["lf", "weno"])
@pytest.mark.parametrize("op", ["mirror_x", "transpose"])
def test_hlld_symmetry_2d(scheme, op):
    m = w.uniform_mesh(2, 16, (2, 2))
    U0 = w.evaluate_on_mesh(m, _ens)

    def to_g(U):
        return np.stack([assemble_uniform(m, U, v) for v in range(9)])

    def from_g(G):
        nb = m.nb
        out = np.empty((m.nleaves, 9, 1, nb, nb))
        for b_, (p, lv, i, j, k) in enumerate(m.leaves):
            out[b_] = G[:, :, j * nb:(j + 1) * nb, i * nb:(i + 1) * nb]
        return out

    def tf(G):
        G = G.copy()
        if op == "mirror_x":
            G = G[..., ::-1].copy(); G[[1, 4]] *= -1
        else:
            G = np.swapaxes(G, 2, 3).copy(); G[[1, 2]] = G[[2, 1]]; G[[4, 5]] = G[[5, 4]]
        return G

    p = dict(scheme=scheme, riemann="hlld", limiter="vanleer")
    a = Oracle(m, U0)
    b = Oracle(m, from_g(tf(to_g(U0))))
    a.advance(p, 3)
    b.advance(p, 3)
    A = tf(to_g(a.get_state()))
    B = to_g(b.get_state())
    for v in range(9):
        assert np.abs(A[v] - B[v]).max() <= 1e-13 * max(np.abs(B[v]).max(), 1e-3), v


@pytest.mark.parametrize("scheme", ["lf", "weno"])
def test_brio_wu_hlld_closer_to_fine_solution_than_hllc(scheme):
    ref = _brio_wu(1536, "weno", "hllc")
    ref200 = ref[0].reshape(192, 8).mean(axis=1)            # 192-cell cell averages
    err = {}
    for rs in ("hllc", "hlld"):
        G = _brio_wu(192, scheme, rs)
        assert np.isfinite(G).all() and (G[0] > 0).all()
        err[rs] = np.abs(G[0] - ref200).mean()
    assert err["hlld"] < 0.9 * err["hllc"], err


@pytest.mark.parametrize("scheme", ["lf", "weno"])
def test_hlld_with_reflux_conserves(scheme):
    mesh = w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.PERIODIC,
                             lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0))
    U0 = w.evaluate_on_mesh(mesh, w.problems.ensemble_problem, seed=5)
    o = Oracle(mesh, U0)
    s0 = o.conservation()
    o.advance(dict(scheme=scheme, riemann="hlld", eglm=0, cp_mode="fixed", cp=0.0), 3)
    s1 = o.conservation()
    assert (np.abs(s1 - s0) / np.maximum(np.abs(s0), 1e-3)).max() <= 2e-14
