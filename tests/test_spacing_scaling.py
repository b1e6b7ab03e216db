"""The step kernel's per-block constants rest on an exact identity of IEEE arithmetic: with
the block spacing computed as the box edge over an integer cell count, dx_L = (hi - lo) /
(nbase nb 2^L) equals dx_0 2^-L, so dt/dx_L equals 2^L dt/dx_0 and its rounding to FP32
equals 2^L times the FP32 rounding of dt/dx_0 (likewise (dt/2)/dx and 2 dx).  Checked here
on random boxes, block edges, levels and time steps, in the same expressions the host and
the finalisation use.
"""

from __future__ import annotations

import numpy as np


def test_level_spacing_and_ratio_scale_exactly():
    rng = np.random.default_rng(1204)
    for _ in range(20000):
        lo = rng.uniform(-3.0, 1.0)
        hi = lo + rng.uniform(1e-3, 50.0)
        nbase = int(rng.integers(1, 64))
        nb = int(rng.choice([8, 16]))
        L = int(rng.integers(0, 13))
        dt = 10.0 ** rng.uniform(-7, -1)
        dx0 = (hi - lo) / float(nbase * nb)
        dxL = (hi - lo) / float((nbase << L) * nb)            # the tree's per-block spacing
        assert dxL == dx0 * 2.0 ** -L
        lam0 = dt / dx0                                       # the finalisation's dt/dx0
        assert dt / dxL == lam0 * 2.0 ** L
        assert (0.5 * dt) / dxL == 0.5 * lam0 * 2.0 ** L
        f32 = np.float32
        assert f32(dt / dxL) == f32(lam0) * f32(2.0 ** L)
        assert f32((0.5 * dt) / dxL) == f32(0.5) * (f32(lam0) * f32(2.0 ** L))
        assert f32(2.0 * dxL) == f32(2.0) * f32(dxL)
        assert f32(0.5 * dt) == f32(0.5) * f32(dt)
