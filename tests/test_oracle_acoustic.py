"""Pins for the oracle's acoustic sweep: m u_tt + damp u_t = L u + src, second-order
leapfrog, zero halo, multilinear source injection and receiver interpolation
(thesis §6.2.1 names this operator, with its sources and receivers, as the
seismic operator the OPS backend could not run; the discrete form is the
standard one).  Pinned by an exact discrete dispersion relation, discrete
energy, a dense brute force, temporal order, interpolation exactness, linearity
and mirror symmetry."""

import math

import numpy as np
import pytest

import fdsynth
from oracle import core, dense


def _mode(shape, k):
    """Π_d sin(k_d π (i_d+1)/(n_d+1)): vanishes on the first zero-halo layer."""
    u = np.ones(())
    lam = 0.0
    for n, kd in zip(shape, k):
        i = np.arange(n)
        u = np.multiply.outer(u, np.sin(kd * math.pi * (i + 1) / (n + 1)))
        lam += -4.0 * math.sin(kd * math.pi / (2 * (n + 1))) ** 2
    return u, lam


@pytest.mark.parametrize("shape,k", [((40, 50), (2, 3)), ((12, 14, 16), (1, 2, 3))])
def test_discrete_dispersion_closed_form(shape, k):
    """Homogeneous m, so = 2: with u^{-1} = cos θ u^0, u^n = cos(nθ) u^0 where
    cos θ = 1 + dt² λ/(2 m h²) and λ h⁻² is the mode's eigenvalue."""
    h, m, dt, nt = 10.0, 1.0 / 2.0 ** 2, 2.0, 300
    u0, lam = _mode(shape, k)
    cth = 1.0 + dt * dt * lam / (h * h) / (2 * m)
    th = math.acos(cth)
    mm = np.full(shape, m)
    u, up, _ = core.acoustic(mm, dt, (h,) * len(shape), 2, nt, u_cur=u0, u_prev=cth * u0)
    assert np.abs(u - math.cos(nt * th) * u0).max() < 1e-11
    assert np.abs(up - math.cos((nt - 1) * th) * u0).max() < 1e-11


def test_temporal_order_two():
    """Against the time-continuous solution cos(ω t) of the same spatial mode,
    the leapfrog error at fixed T falls by 4 when dt halves."""
    shape, k, h, m = (30, 34), (2, 1), 10.0, 0.25
    u0, lam = _mode(shape, k)
    omega = math.sqrt(-lam / (h * h) / m)
    T = 400.0
    errs = []
    for nt in (200, 400, 800):
        dt = T / nt
        u, _, _ = core.acoustic(np.full(shape, m), dt, (h, h), 2, nt, u_cur=u0,
                                u_prev=math.cos(omega * dt) * u0)
        errs.append(np.abs(u - math.cos(omega * T) * u0).max())
    for a, b in zip(errs, errs[1:]):
        assert abs(a / b - 4.0) < 0.1, errs


def _energy(u_new, u_old, m, dt, h, so):
    lap = core.laplacian(u_old, h, so)
    return float(np.sum(m * ((u_new - u_old) / dt) ** 2) - np.sum(u_new * lap))


@pytest.mark.parametrize("so", (2, 8, 16))
def test_discrete_energy_conserved_without_damping(so):
    rng = np.random.default_rng(so)
    shape, h = (14, 15, 16), (10.0,) * 3
    m = rng.uniform(1 / 4.5 ** 2, 1 / 1.5 ** 2, shape)
    u = rng.standard_normal(shape)
    up = u + 0.1 * rng.standard_normal(shape)
    dt = 0.3 * 10.0 / 4.5
    e0 = _energy(u, up, m, dt, h, so)
    for _ in range(5):
        u, up, _ = core.acoustic(m, dt, h, so, 20, u_cur=u, u_prev=up)
        assert abs(_energy(u, up, m, dt, h, so) - e0) < 1e-11 * abs(e0)


def test_discrete_energy_decreases_with_damping():
    rng = np.random.default_rng(11)
    shape, h = (20, 22), (10.0, 10.0)
    m = rng.uniform(0.05, 0.4, shape)
    damp = rng.uniform(0.0, 0.02, shape)
    u = rng.standard_normal(shape)
    up = u.copy()
    dt = 1.2
    e = _energy(u, up, m, dt, h, 4)
    for _ in range(10):
        u, up, _ = core.acoustic(m, dt, h, 4, 3, damp=damp, u_cur=u, u_prev=up)
        e_new = _energy(u, up, m, dt, h, 4)
        assert e_new <= e + 1e-12 * abs(e)
        e = e_new


@pytest.mark.parametrize("so", (2, 4, 6, 8, 10, 12, 14, 16))
@pytest.mark.parametrize("shape", [(5, 6, 7), (6, 9), (2, 3, 2)])
def test_matches_dense_brute_force(so, shape):
    rng = np.random.default_rng(so + 7 * len(shape))
    nd = len(shape)
    m = rng.uniform(0.05, 0.45, shape)
    damp = rng.uniform(0.0, 0.05, shape)
    u = rng.standard_normal(shape)
    up = rng.standard_normal(shape)
    h = tuple(rng.uniform(8, 12, nd))
    ext = [(n - 1) * hd for n, hd in zip(shape, h)]
    sc = rng.uniform(0, 1, (3, nd)) * ext
    sc[1] = sc[0]                                       # two sources on one spot
    rc = np.vstack([rng.uniform(0, 1, (4, nd)) * ext, np.array([ext]), np.zeros((1, nd))])
    wav = rng.standard_normal((12, 3))
    args = dict(damp=damp, u_cur=u, u_prev=up, src_coords=sc, wavelet=wav, rec_coords=rc, n0=2)
    a = core.acoustic(m, 0.8, h, so, 9, **args)
    b = dense.acoustic(m, 0.8, h, so, 9, **args)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-12 * max(1.0, np.abs(y).max())


@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 6)])
def test_corners_match_tent_functions_and_reproduce_linear_data(shape):
    rng = np.random.default_rng(2)
    nd = len(shape)
    h = tuple(rng.uniform(5, 15, nd))
    ext = np.array([(n - 1) * hd for n, hd in zip(shape, h)])
    pts = list(rng.uniform(0, 1, (20, nd)) * ext) + [ext, np.zeros(nd), ext * 0.5]
    coef = rng.standard_normal(nd)
    grid = np.meshgrid(*[np.arange(n) * hd for n, hd in zip(shape, h)], indexing="ij")
    lin = (3.0 + sum(c * g for c, g in zip(coef, grid))).reshape(-1)
    for p in pts:
        node, wt = core.corners(shape, h, p)
        row = np.zeros(int(np.prod(shape)))
        np.add.at(row, node, wt)
        assert np.abs(row - dense.tent_row(shape, h, p)).max() < 1e-14
        assert abs(wt.sum() - 1.0) < 1e-14 and wt.min() >= 0
        assert abs(row @ lin - (3.0 + coef @ p)) < 1e-11


def test_coordinates_outside_the_grid_are_rejected():
    for bad in ([-0.1, 5.0], [5.0, 60.01], [float("nan"), 1.0]):
        with pytest.raises(core.OracleError):
            core.corners((6, 7), (10.0, 10.0), bad)


def test_injection_interpolation_adjoint():
    """<P^T s, u> = <s, P u>: the scatter one step of injection performs (read off
    the oracle as u^{1} - u^{1}|no source, scaled back by dt²/m) against the
    oracle's interpolation of a random field at the same points."""
    rng = np.random.default_rng(9)
    shape, h, dt = (7, 8, 9), (10.0,) * 3, 1.0
    m = rng.uniform(0.1, 0.4, shape)
    pts = fdsynth.random_points(shape, h, 5, seed=4).astype(np.float64)
    s = rng.standard_normal((1, 5))
    z = np.zeros(shape)
    with_src, _, _ = core.acoustic(m, dt, h, 4, 1, u_cur=z, u_prev=z, src_coords=pts, wavelet=s)
    pts_u = with_src * m / (dt * dt)                       # = P^T s
    u = rng.standard_normal(shape)
    _, _, rec = core.acoustic(m, dt, h, 4, 0, u_cur=u, rec_coords=pts)   # rec[0] = P u
    assert abs(np.sum(pts_u * u) - np.sum(s[0] * rec[0])) < 1e-12 * np.abs(u).sum()


def test_traces_linear_in_wavelet():
    p = fdsynth.acoustic_problem(n=24, ndim=3, so=4, nbl=6, nt=40, nrec=8, seed=3)
    args = dict(damp=p["damp"], src_coords=p["src_coords"], rec_coords=p["rec_coords"])
    _, _, r1 = core.acoustic(p["m"], p["dt"], p["spacing"], 4, 40, wavelet=p["wavelet"], **args)
    _, _, r2 = core.acoustic(p["m"], p["dt"], p["spacing"], 4, 40, wavelet=2 * p["wavelet"].astype(np.float64), **args)
    assert np.abs(r2 - 2 * r1).max() < 1e-12 * np.abs(r1).max()
    assert np.abs(r1).max() > 0


def test_mirror_symmetric_traces():
    """Centred source in a model that depends on depth only: receivers placed
    symmetrically about the centre along x record identical traces."""
    n, h = 25, 10.0
    shape = (n, n, n)
    v = np.broadcast_to(np.linspace(1.5, 3.0, n).reshape(n, 1, 1), shape)
    m = 1.0 / v ** 2
    c = (n - 1) * h / 2
    src = np.array([[c, c, c]])
    rec = np.array([[c + 30, c, c - 47.0], [c + 30, c, c + 47.0], [c + 30, c - 47, c], [c + 30, c + 47, c]])
    wav = fdsynth.ricker(60, 1.0, 0.03).reshape(-1, 1)
    _, _, r = core.acoustic(m, 1.0, (h,) * 3, 8, 60, src_coords=src, wavelet=wav, rec_coords=rec)
    scale = np.abs(r).max()
    assert scale > 0
    assert np.abs(r[:, 0] - r[:, 1]).max() < 1e-12 * scale
    assert np.abs(r[:, 2] - r[:, 3]).max() < 1e-12 * scale
    assert np.abs(r[:, 0] - r[:, 2]).max() < 1e-12 * scale     # x <-> y symmetry as well


def test_chunked_run_equals_single_run():
    p = fdsynth.acoustic_problem(n=20, ndim=2, so=8, nbl=4, nt=30, nrec=5, seed=1)
    args = dict(damp=p["damp"], src_coords=p["src_coords"], wavelet=p["wavelet"], rec_coords=p["rec_coords"])
    u, up, r = core.acoustic(p["m"], p["dt"], p["spacing"], 8, 30, **args)
    u1, up1, ra = core.acoustic(p["m"], p["dt"], p["spacing"], 8, 12, **args)
    u2, up2, rb = core.acoustic(p["m"], p["dt"], p["spacing"], 8, 18, u_cur=u1, u_prev=up1, n0=12, **args)
    assert np.array_equal(u, u2) and np.array_equal(up, up2)
    assert np.array_equal(r, np.vstack([ra, rb[1:]]))


def test_wavelet_too_short_is_rejected():
    m = np.ones((5, 5))
    with pytest.raises(core.OracleError):
        core.acoustic(m, 0.1, (1.0, 1.0), 2, 5, src_coords=[[1.0, 1.0]], wavelet=np.zeros((4, 1)))
