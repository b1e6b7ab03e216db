"""Oracle pins for thermal conduction with its subcycle (Sec. 3.6; the Sec. 5 conduction test).

The energy update e_i += h/dx^2 (sqrt(k_i k_i+1)(T_i+1 - T_i) - sqrt(k_i k_i-1)(T_i - T_i-1)),
kappa = kappa0 T^(5/2), its time step c_cfl min(dx)^2/(n_dim max(kappa T/p)), and the
field-aligned form div(kappa (b.grad T) b) are pinned against what the mathematics fixes:
* a small-amplitude temperature mode decays by exactly the factor the discrete linear theory
  gives per substep, in every direction and dimension, and along B by that factor times
  cos^2 of the field angle (not at all across B);
* a uniform temperature stays bit for bit; a clipped gradient gives the clipped flux;
* the energy total holds to round-off on periodic meshes, and on AMR with the energy reflux;
* the conduction time step matches its closed form, and bounds dt without the subcycle;
* with and without the subcycle the temperature differs by less than 0.5 % (the paper's
  Sec. 5 comparison), with the subcycle taking several substeps per step.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import workloads as w
from workloads.problems import conserved_from_primitive
from oracle import Oracle
from tests.helpers import assemble_uniform, run_to_time

GAMMA = 5.0 / 3.0


def _temperature(U, gamma=GAMMA):
    rho = U[:, 0]
    p = (gamma - 1.0) * (U[:, 7] - 0.5 * (U[:, 1] ** 2 + U[:, 2] ** 2 + U[:, 3] ** 2) / rho
                         - 0.5 * (U[:, 4] ** 2 + U[:, 5] ** 2 + U[:, 6] ** 2))
    return np.maximum(p, 0.0) / rho


def _mode_mesh(ndim, axis, n=64, nb=16):
    nbase = [1, 1, 1][:ndim]
    nbase[axis] = n // nb
    lo, hi = [0.0, 0.0, 0.0], [1.0, 1.0, 1.0]
    for d in range(ndim):
        if d != axis:
            hi[d] = nb / n                                   # one block across: square cells
    return w.uniform_mesh(ndim, nb, nbase, lo=tuple(lo), hi=tuple(hi))


def _mode_state(mesh, axis, eps, B=(0.0, 0.0, 0.0), T0=1.0, rho=1.0):
    def ic(X, Y, Z, **_):
        x = (X, Y, Z)[axis]
        T = T0 * (1.0 + eps * np.cos(2 * math.pi * x))
        return conserved_from_primitive(rho + 0 * X, 0.0, 0.0, 0.0, B[0], B[1], B[2], rho * T, GAMMA)
    return w.evaluate_on_mesh(mesh, ic)


def _mode_amplitude(mesh, U, axis):
    T = _temperature(U)
    xs = []
    for b in range(mesh.nleaves):
        X, Y, Z = w.problems.cell_centres(mesh, b)
        xs.append((X, Y, Z)[axis])
    x = np.stack(xs)
    T = T.reshape(x.shape)
    return 2.0 * np.mean((T - T.mean()) * np.cos(2 * math.pi * x))


@pytest.mark.parametrize("ndim,axis", [(2, 0), (2, 1), (3, 2)])
def test_isotropic_mode_decays_by_the_discrete_factor(ndim, axis):
    mesh = _mode_mesh(ndim, axis)
    eps, kappa0, rho, dt = 1e-6, 0.01, 1.0, 0.5
    U0 = _mode_state(mesh, axis, eps)
    o = Oracle(mesh, U0)
    p = dict(conduction="isotropic", kappa0=kappa0, c_cfl=0.4)
    assert o.conduct(p, dt) == 0
    dx = 1.0 / 64
    kap = kappa0                                            # T0 = 1
    dtc = 0.4 * dx * dx / (ndim * kap / rho)
    n = math.ceil(dt / dtc)
    h = dt / n
    g = 1.0 - (GAMMA - 1.0) * h * kap / (rho * dx * dx) * 4.0 * math.sin(math.pi * dx) ** 2
    got = _mode_amplitude(mesh, o.get_state(), axis) / _mode_amplitude(mesh, U0, axis)
    assert abs(got - g ** n) <= 1e-5 * g ** n, (got, g ** n)
    assert g ** n < 0.95                                    # the mode really decayed


@pytest.mark.parametrize("theta", [0.0, 30.0, 90.0])
def test_aligned_mode_decays_by_cos2_of_the_field_angle(theta):
    mesh = _mode_mesh(2, 0)
    eps, kappa0, rho, dt = 1e-6, 0.01, 1.0, 0.5
    th = math.radians(theta)
    U0 = _mode_state(mesh, 0, eps, B=(math.cos(th), math.sin(th), 0.0))
    o = Oracle(mesh, U0)
    assert o.conduct(dict(conduction="aligned", kappa0=kappa0, c_cfl=0.4), dt) == 0
    if theta == 90.0:
        np.testing.assert_array_equal(o.get_state(), U0)    # heat does not cross B
        return
    dx = 1.0 / 64
    dtc = 0.4 * dx * dx / (2 * kappa0 / rho)
    n = math.ceil(dt / dtc)
    h = dt / n
    c2 = math.cos(th) ** 2
    g = 1.0 - (GAMMA - 1.0) * h * kappa0 * c2 / (rho * dx * dx) * 4.0 * math.sin(math.pi * dx) ** 2
    got = _mode_amplitude(mesh, o.get_state(), 0) / _mode_amplitude(mesh, U0, 0)
    assert abs(got - g ** n) <= 1e-5 * g ** n, (got, g ** n)


@pytest.mark.parametrize("mode", ["isotropic", "aligned"])
def test_uniform_temperature_unchanged(mode):
    mesh = w.uniform_mesh(2, 8, (2, 2))
    U0 = w.evaluate_on_mesh(mesh, w.problems.uniform_state)
    o = Oracle(mesh, U0)
    o.conduct(dict(conduction=mode, kappa0=0.05), 0.3)
    np.testing.assert_array_equal(o.get_state(), U0)


def test_clipped_gradient_gives_the_clipped_flux():
    mesh = w.uniform_mesh(2, 8, (2, 1), hi=(1.0, 0.5, 1.0))
    def ic(X, Y, Z, **_):
        T = np.where(X < 0.5, 1.0, 2.0)
        return conserved_from_primitive(1.0 + 0 * X, 0, 0, 0, 0, 0, 0, T, GAMMA)
    U0 = w.evaluate_on_mesh(mesh, ic)
    o = Oracle(mesh, U0)
    gmax, kappa0, dt = 0.5, 1e-3, 1e-4
    o.conduct(dict(conduction="isotropic", kappa0=kappa0, grad_t_max=gmax), dt)
    dE = o.get_state()[:, 7] - U0[:, 7]
    dx = 1.0 / 16
    kf = kappa0 * math.sqrt(1.0 * 2.0 ** 2.5)               # geometric mean of kappa(1), kappa(2)
    q = dt * kf * gmax / dx
    # the cells on either side of the two jumps (x = 0.5 and the periodic x = 0) move by q
    E = np.concatenate([dE[0, 0], dE[1, 0]], axis=1)[0]
    # dE is the difference of two energies near 1.5: exact to a few ulp of 1.5
    np.testing.assert_allclose(E[[7, 8]], [q, -q], rtol=0, atol=1e-15)
    np.testing.assert_allclose(E[[0, 15]], [q, -q], rtol=0, atol=1e-15)
    assert np.all(E[1:7] == 0) and np.all(E[9:15] == 0)


def _mixed_T(mesh):
    def ic(X, Y, Z, **_):
        T = 1.0 + 0.5 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * (Y + Z))
        return conserved_from_primitive(1.0 + 0.3 * np.cos(2 * math.pi * Y), 0, 0, 0, 0.6, 0.3, 0.2 + 0 * X,
                                        T * (1.0 + 0.3 * np.cos(2 * math.pi * Y)), GAMMA)
    return w.evaluate_on_mesh(mesh, ic)


@pytest.mark.parametrize("mode", ["isotropic", "aligned"])
@pytest.mark.parametrize("amr", [False, True])
def test_energy_total_conserved(mode, amr):
    if amr:
        mesh = w.radial_amr_mesh(2, 8, (2, 2), 2, radii=(0.16, 0.34), bc=w.mesh.PERIODIC,
                                 lo=(0, 0, 0), hi=(1, 1, 1), centre=(0.5, 0.5, 0))
    else:
        mesh = w.uniform_mesh(3, 8, (2, 2, 2))
    U0 = _mixed_T(mesh)
    drift = {}
    for rf in ((0, 1) if amr else (1,)):
        o = Oracle(mesh, U0)
        e0 = o.conservation()[0, 7]
        o.conduct(dict(conduction=mode, kappa0=0.02, reflux=rf), 0.05)
        e1 = o.conservation()[0, 7]
        drift[rf] = abs(e1 - e0) / abs(e0)
        assert not np.array_equal(o.get_state(), U0)
    assert drift[1] <= 1e-14, drift
    if amr:
        assert drift[0] >= 1e-9, drift


def test_conduction_time_step_closed_form():
    mesh = w.uniform_mesh(2, 16, (2, 2))
    U0 = _mixed_T(mesh)
    kappa0, c_cfl = 0.02, 0.4
    o = Oracle(mesh, U0)
    o.fill_ghosts()
    dt_sub = o.cfl(dict(conduction="isotropic", kappa0=kappa0, subcycle=1, c_cfl=c_cfl))[0]
    T = _temperature(U0)
    dx = 1.0 / 32
    ref = c_cfl * dx * dx / (2 * np.max(kappa0 * T ** 2.5 / U0[:, 0]))
    assert abs(o.dtc()[0] - ref) <= 1e-14 * ref
    o2 = Oracle(mesh, U0)
    o2.fill_ghosts()
    dt_nosub = o2.cfl(dict(conduction="isotropic", kappa0=kappa0, subcycle=0, c_cfl=c_cfl))[0]
    assert dt_nosub == min(dt_sub, o.dtc()[0])
    assert ref < dt_sub                                      # conduction is the stiffer limit here


def _x8_like():
    """The oblique-field conduction test's parameters (kappa0 = 0.001, rho = 0.1, p = 0.1,
    B = (1, 1, 0), a hot region with rho = 0.025 -> T = 4), in a periodic box."""
    mesh = w.uniform_mesh(2, 16, (4, 4), lo=(-0.5, -0.5, 0), hi=(0.5, 0.5, 1))

    def ic(X, Y, Z, **_):
        hot = (np.abs(X) < 0.1) & (np.abs(Y) < 0.1)
        rho = np.where(hot, 0.025, 0.1)
        return conserved_from_primitive(rho, 0, 0, 0, 1.0, 1.0, 0.0, 0.1, GAMMA)
    return mesh, w.evaluate_on_mesh(mesh, ic)


def test_subcycle_matches_no_subcycle_within_half_a_percent():
    mesh, U0 = _x8_like()
    base = dict(gamma=GAMMA, scheme="weno", conduction="aligned", kappa0=1e-3, c_cfl=0.4)
    out, steps = {}, {}
    for sub in (1, 0):
        o = Oracle(mesh, U0)
        steps[sub] = run_to_time(o, dict(base, subcycle=sub), 0.01)
        out[sub] = _temperature(o.get_state())
        if sub:
            o.fill_ghosts()
            o.cfl(dict(base, subcycle=1))
            assert o.speeds()[0, 0] / o.dtc()[0] >= 5.0      # several substeps per step
    T0 = _temperature(U0)
    assert np.abs(out[1] - T0).max() > 0.05 * T0.max()      # heat has moved
    assert np.abs(out[1] - out[0]).max() <= 0.005 * out[0].max()
    assert steps[0] > 3 * steps[1]
