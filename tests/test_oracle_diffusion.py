"""Pins for the oracle's diffusion sweep (thesis §5.1.2: u_t = ν(u_xx + u_yy),
forward Euler, time order 1; interior-only update as in §2.1.1's
``subdomain=grid.interior``).  Checked against the exact per-step decay of a
sine mode, a dense-matrix brute force and invariants."""

import math

import numpy as np
import pytest

import fdsynth
from oracle import core, dense


def _sine_mode(n, ndim, k=(1, 1, 1)):
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    u = np.ones(())
    for d in range(ndim):
        s = np.sin(k[d] * math.pi * x)
        s[0] = s[-1] = 0.0
        u = np.multiply.outer(u, s)
    return u, h


@pytest.mark.parametrize("ndim,n,k", [(2, 128, (1, 1)), (2, 33, (3, 2)), (3, 24, (1, 2, 3))])
def test_sine_mode_decays_by_exact_discrete_factor(ndim, n, k):
    """Π sin(k_d π x_d) is an eigenvector of the so=2 interior update with zero
    boundary nodes: u^n = g^n u^0, g = 1 + ν dt Σ_d (-4/h²) sin²(k_d π h/2)."""
    u0, h = _sine_mode(n, ndim, k)
    nu, nt = 0.5, 100
    dt = 0.2 * h * h / nu / ndim * 2
    g = 1.0 + nu * dt * sum(-4.0 / h ** 2 * math.sin(kd * math.pi * h / 2) ** 2 for kd in k[:ndim])
    u = core.diffusion(u0, (h,) * ndim, 2, nu, dt, nt)
    assert np.abs(u - g ** nt * u0).max() < 1e-13


def test_benchmark_problem_decay_value():
    """128² nodes on [0,1]², ν = 0.5, ν dt/h² = 0.2, 100 steps: g = 1 - 1.6 sin²(πh/2)
    with h = 1/127, so g^100 = 0.9758187512772...; the continuum decay
    exp(-2π²ν t) differs from it in the sixth digit, which this pin can see."""
    u0, h = _sine_mode(128, 2)
    dt = 0.2 * h * h / 0.5
    u = core.diffusion(u0, (h, h), 2, 0.5, dt, 100)
    ratio = u[64, 40] / u0[64, 40]
    assert abs(ratio - 0.97581875127726) < 1e-12
    assert abs(ratio - math.exp(-2 * math.pi ** 2 * 0.5 * 100 * dt)) > 1e-7


def test_fp32_problem_matches_fp64_mode():
    """The float32 inputs of the benchmark problem stay within float32 rounding of the mode."""
    p = fdsynth.diffusion_problem(128)
    u0, h = _sine_mode(128, 2)
    assert np.abs(p["u0"].astype(np.float64) - u0).max() < 1e-7
    assert p["u0"][0].max() == 0 and p["u0"][:, -1].max() == 0


@pytest.mark.parametrize("so", (2, 4, 8, 16))
@pytest.mark.parametrize("shape", [(7, 9), (1, 5), (3, 3), (5, 6, 7), (3, 4, 3)])
def test_matches_dense_brute_force(so, shape):
    rng = np.random.default_rng(so * 100 + len(shape))
    u0 = rng.standard_normal(shape)
    spacing = tuple(rng.uniform(0.2, 0.4, len(shape)))
    a = core.diffusion(u0, spacing, so, 0.7, 0.003, 6)
    b = dense.diffusion(u0, spacing, so, 0.7, 0.003, 6)
    assert np.abs(a - b).max() < 1e-12


def test_boundary_nodes_are_held_and_nt0_is_identity():
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((6, 7, 8))
    u = core.diffusion(u0, (0.3,) * 3, 4, 0.5, 0.001, 5)
    for d in range(3):
        for i in (0, u0.shape[d] - 1):
            sl = [slice(None)] * 3
            sl[d] = i
            assert np.array_equal(u[tuple(sl)], u0[tuple(sl)])
    assert np.array_equal(core.diffusion(u0, (0.3,) * 3, 4, 0.5, 0.001, 0), u0)


def test_maximum_principle():
    """ν dt Σ 1/h² ≤ 1/2 with so=2: the update is a convex combination, so
    values stay within the initial range."""
    rng = np.random.default_rng(5)
    u0 = rng.uniform(-1, 1, (20, 20))
    u = core.diffusion(u0, (1.0, 1.0), 2, 1.0, 0.25, 50)
    assert u.max() <= u0.max() + 1e-15 and u.min() >= u0.min() - 1e-15


def test_bad_arguments_raise():
    with pytest.raises(ValueError):
        core.diffusion(np.zeros((4, 4)), (1.0, 1.0), 3, 0.5, 0.1, 1)
    with pytest.raises(core.OracleError):           # odd order with explicit weights
        core.diffusion(np.zeros((4, 4)), (1.0, 1.0), 3, 0.5, 0.1, 1, weights=[-2.0, 1.0])
    with pytest.raises(core.OracleError):
        core.diffusion(np.zeros((4, 4)), (1.0, 1.0), 2, 0.5, 0.1, -1)
