"""Pins for the oracle's FWI gradient (adjoint-state method of the discrete
leapfrog): it equals central finite differences of the oracle's objective J at
every model point, in 2-D and 3-D, with damping everywhere (so the source-node
term that vanishes where damp = 0 is exercised) -- an independent route to the
same derivative."""

import numpy as np
import pytest

from oracle import core, fwi


def _case(shape, so, nt, seed):
    rng = np.random.default_rng(seed)
    nd = len(shape)
    h = (10.0,) * nd
    m = rng.uniform(1 / 3.0 ** 2, 1 / 1.8 ** 2, shape)
    damp = rng.uniform(0.0, 0.02, shape)
    dt = 1.2
    ext = np.array([(n - 1) * 10.0 for n in shape])
    src = rng.uniform(0.2, 0.8, (2, nd)) * ext
    rec = rng.uniform(0.0, 1.0, (5, nd)) * ext
    wav = rng.standard_normal((nt, 2))
    d_obs = rng.standard_normal((nt + 1, 5)) * 1e-3
    return m, damp, dt, h, src, wav, rec, d_obs


@pytest.mark.parametrize("shape,so", [((7, 8), 4), ((4, 5, 6), 2), ((5, 5, 4), 8)])
def test_gradient_matches_finite_differences(shape, so):
    nt = 14
    m, damp, dt, h, src, wav, rec, d_obs = _case(shape, so, nt, seed=len(shape) + so)
    J, g = fwi.gradient(m, damp, dt, h, so, nt, src, wav, rec, d_obs)
    J0, _ = fwi.objective(m, damp, dt, h, so, nt, src, wav, rec, d_obs)
    assert abs(J - J0) <= 1e-12 * abs(J0)
    fd = np.zeros_like(m)
    for i in range(m.size):
        e = np.zeros(m.size)
        eps = 1e-6 * m.reshape(-1)[i]
        e[i] = eps
        e = e.reshape(m.shape)
        jp, _ = fwi.objective(m + e, damp, dt, h, so, nt, src, wav, rec, d_obs)
        jm, _ = fwi.objective(m - e, damp, dt, h, so, nt, src, wav, rec, d_obs)
        fd.reshape(-1)[i] = (jp - jm) / (2 * eps)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(g - fd).max() <= 1e-6 * scale


def test_zero_residual_gives_zero_gradient():
    m, damp, dt, h, src, wav, rec, _ = _case((6, 7), 4, 10, seed=3)
    _, d = fwi.objective(m, damp, dt, h, 4, 10, src, wav, rec, np.zeros((11, 5)))
    J, g = fwi.gradient(m, damp, dt, h, 4, 10, src, wav, rec, d)
    Jr, gr = fwi.gradient(m, damp, dt, h, 4, 10, src, wav, rec, d + 1e-3)
    assert J < 1e-25 and np.abs(g).max() <= 1e-12 * np.abs(gr).max()

