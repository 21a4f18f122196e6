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


# ----------------------------------------------------------------------------
# Odd-reflection boundary mode: values outside the grid are the negated mirror
# images about the boundary nodes, which makes every sine mode an exact
# eigenvector of the interior update at every space order.
# ----------------------------------------------------------------------------
def _odd_factor(so, n, ndim, k, nu, dt):
    """Exact per-step factor of Π sin(k_d π x_d) under the odd-reflection update:
    1 + ν dt Σ_d (w_0 + 2 Σ_j w_j cos(j k_d π h)) / h²  (h = 1/(n-1))."""
    from oracle.weights import fd_weights
    w = [float(x) for x in fd_weights(so)]
    h = 1.0 / (n - 1)
    lam = sum((w[0] + 2.0 * sum(w[j] * math.cos(j * kd * math.pi * h)
                                for j in range(1, so // 2 + 1))) / (h * h) for kd in k[:ndim])
    return 1.0 + nu * dt * lam


@pytest.mark.parametrize("so", (2, 4, 6, 8, 10, 12, 14, 16))
@pytest.mark.parametrize("ndim,n,k", [(2, 41, (1, 1)), (2, 30, (2, 3)), (3, 19, (1, 2, 1))])
def test_odd_reflection_sine_mode_decays_by_exact_factor(so, ndim, n, k):
    u0, h = _sine_mode(n, ndim, k)
    nu, nt = 0.5, 40
    dt = 0.05 * h * h / nu
    g = _odd_factor(so, n, ndim, k, nu, dt)
    u = core.diffusion(u0, (h,) * ndim, so, nu, dt, nt, boundary="odd")
    assert np.abs(u - g ** nt * u0).max() < 1e-13
    if so > 2:   # the zero halo breaks the eigenvector property above so = 2
        z = core.diffusion(u0, (h,) * ndim, so, nu, dt, nt)
        assert np.abs(z - g ** nt * u0).max() > 1e-9


def test_odd_reflection_equals_zero_halo_at_second_order():
    """At so = 2 the node next to a boundary reaches only the boundary node."""
    rng = np.random.default_rng(11)
    u0 = rng.standard_normal((9, 10, 11))
    for d in range(3):
        for i in (0, u0.shape[d] - 1):
            sl = [slice(None)] * 3
            sl[d] = i
            u0[tuple(sl)] = 0.0
    a = core.diffusion(u0, (0.3, 0.25, 0.2), 2, 0.5, 0.002, 7, boundary="odd")
    b = core.diffusion(u0, (0.3, 0.25, 0.2), 2, 0.5, 0.002, 7)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("so", (4, 8, 12))
@pytest.mark.parametrize("shape", [(9, 11), (7, 8, 9)])
def test_odd_reflection_matches_dense_brute_force(so, shape):
    rng = np.random.default_rng(so + len(shape))
    u0 = rng.standard_normal(shape)
    spacing = tuple(rng.uniform(0.2, 0.4, len(shape)))
    if max(shape) - 1 < so // 2 or min(shape) - 1 < so // 2:
        pytest.skip("grid too small for the mirror")
    a = core.diffusion(u0, spacing, so, 0.7, 0.002, 5, boundary="odd")
    b = dense.diffusion(u0, spacing, so, 0.7, 0.002, 5, boundary="odd")
    assert np.abs(a - b).max() < 1e-12


def test_odd_reflection_needs_room_for_the_mirror():
    with pytest.raises(core.OracleError):
        core.diffusion(np.zeros((5, 9)), (1.0, 1.0), 10, 0.5, 0.01, 1, boundary="odd")


# --- every node updated (§2.1.1's operator without the grid.interior subdomain) ---

@pytest.mark.parametrize("ndim,n,k", [(2, 40, (1, 1)), (2, 31, (3, 2)), (3, 18, (1, 2, 3))])
def test_all_node_update_sine_mode_decays_by_exact_factor(ndim, n, k):
    """Every node updated with zero values outside: the mode Π sin(k_d π (i+1)/(n+1)),
    i = 0..n-1, vanishes on the first outside layer, so at so 2 it is an exact
    eigenvector: u^n = g^n u^0 with g = 1 + ν dt Σ_d (-4/h²) sin²(k_d π / (2(n+1)))."""
    h = 1.0 / (n + 1)
    u0 = np.ones(())
    for d in range(ndim):
        u0 = np.multiply.outer(u0, np.sin(k[d] * math.pi * (np.arange(n) + 1) / (n + 1)))
    nu, nt = 0.5, 80
    dt = 0.1 * h * h / nu
    g = 1.0 + nu * dt * sum(-4.0 / h ** 2 * math.sin(kd * math.pi / (2 * (n + 1))) ** 2
                            for kd in k[:ndim])
    u = core.diffusion(u0, (h,) * ndim, 2, nu, dt, nt, interior=False)
    assert np.abs(u - g ** nt * u0).max() < 1e-13
    # the interior update holds the boundary nodes instead: a different sweep
    assert np.abs(core.diffusion(u0, (h,) * ndim, 2, nu, dt, nt) - u).max() > 1e-3


@pytest.mark.parametrize("so", (2, 4, 8, 12, 16))
@pytest.mark.parametrize("shape", [(9, 11), (6, 7, 8)])
def test_all_node_update_matches_dense_brute_force(so, shape):
    rng = np.random.default_rng(so + len(shape))
    u0 = rng.standard_normal(shape)
    h = tuple(1.0 / (n + 1) for n in shape)
    nu = 0.5
    dt = 0.02 * min(h) ** 2
    got = core.diffusion(u0, h, so, nu, dt, 12, interior=False)
    ref = dense.diffusion(u0, h, so, nu, dt, 12, interior_only=False)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    edge = got[0]
    assert np.abs(edge - u0[0]).max() > 0          # boundary nodes move


def test_odd_reflection_needs_the_interior_update():
    u0 = np.ones((12, 12))
    with pytest.raises(core.OracleError):
        core.diffusion(u0, (0.1, 0.1), 4, 0.5, 1e-4, 1, boundary="odd", interior=False)
