"""The interface fluxes under an exchange of coordinate axes (the step kernel computes a y face
as the x-face flux of the state with the x and y components of m and B exchanged, then
exchanges the result back).  For the exchange P of x and y, F_y(U) = P F_x(P U) holds bitwise
for the physical flux, the Rusanov flux f_m and HLLC: the exchange only swaps the first two
terms of the sums it reorders (|m|^2, |B|^2, v.B), and a + b = b + a in IEEE arithmetic.  For
the exchange of x and z the identity holds mathematically but reorders three-term sums, so it
holds to rounding only -- the reason the kernel keeps its own z-direction flux code.
"""

from __future__ import annotations

import numpy as np
import pytest

from workloads.problems import conserved_from_primitive
from oracle import oracle as O

G53 = 5.0 / 3.0
MX, MY, MZ, BX, BY, BZ = 1, 2, 3, 4, 5, 6


def _exchange(w, d):
    """x and d components of m and B exchanged (d = 1: y, d = 2: z)."""
    w = np.array(w, dtype=np.float64)
    w[[MX, MX + d]] = w[[MX + d, MX]]
    w[[BX, BX + d]] = w[[BX + d, BX]]
    return w


def _state(rng):
    rho = rng.uniform(0.2, 3.0)
    v = rng.uniform(-2.0, 2.0, 3)
    B = rng.uniform(-1.5, 1.5, 3)
    p = rng.uniform(0.05, 2.0)
    return np.array(conserved_from_primitive(rho, v[0], v[1], v[2], B[0], B[1], B[2], p, G53,
                                             rng.uniform(-0.2, 0.2)), dtype=np.float64).reshape(9)


FLUXES = {
    "physical": lambda d, a, b, ch: O.flux(d, a, G53, ch),
    "rusanov": lambda d, a, b, ch: O.lf_flux(d, a, b, G53, ch),
    "hllc": lambda d, a, b, ch: O.hllc_flux(d, a, b, G53, ch),
}


@pytest.mark.parametrize("kind", list(FLUXES))
def test_y_flux_is_the_exchanged_x_flux_bitwise(kind):
    f = FLUXES[kind]
    rng = np.random.default_rng(1204)
    for _ in range(300):
        a, b, ch = _state(rng), _state(rng), rng.uniform(0.5, 4.0)
        direct = f(1, a, b, ch)
        via_x = _exchange(f(0, _exchange(a, 1), _exchange(b, 1), ch), 1)
        np.testing.assert_array_equal(direct, via_x)


@pytest.mark.parametrize("kind", list(FLUXES))
def test_z_flux_is_the_exchanged_x_flux_to_rounding(kind):
    f = FLUXES[kind]
    rng = np.random.default_rng(5849)
    exact = 0
    for _ in range(300):
        a, b, ch = _state(rng), _state(rng), rng.uniform(0.5, 4.0)
        direct = f(2, a, b, ch)
        via_x = _exchange(f(0, _exchange(a, 2), _exchange(b, 2), ch), 2)
        scale = np.maximum(np.abs(direct), 1.0)
        assert np.max(np.abs(direct - via_x) / scale) <= 1e-13
        exact += int(np.array_equal(direct, via_x))
    assert exact < 300                                       # reordered sums round differently
