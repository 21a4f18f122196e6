"""Parity at full benchmark sizes, in the launch configurations bench.py times.

* 256³ so 8 shot (damping layer 40, layered model, Ricker source at the centre,
  256 receivers, 500 steps) against one FP64 oracle run on the whole grid: the
  wavefield and the traces within 1e-4 relative L2, for the default 32-wide
  tile, the tile bench.py's autotuner picked on the B300 (64 x 32 x-pair tiles,
  64-plane segments, 1 CTA per SM, whole-segment split), the same with the C
  tile skipped on undamped tile-planes, and whatever the autotuner picks on the
  box the test runs on.
* 512³ at so 4/8/12/16: one step from random fields, checked on sampled points
  (random, grid corners, tile and z-block seams) against the oracle evaluated
  point by point on (2R+1)³ windows, with the default tile and with the tile the
  autotuner picks (the bench's sweep configuration: on the B300 the x-pair work
  queue, 24-row tiles at so 12/16); 20 steps at so 8 and 16 against the oracle on
  the whole grid, the tuned tile bitwise the default one; the 512³ diffusion step
  (so 4/8/16, tuned tile) on sampled points.
"""

import numpy as np
import pytest

import fdsynth
from helpers import rel_l2
from oracle import core as oracle

pytestmark = pytest.mark.gpu

TOL_WAVE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


# The tile the bench's autotuner chose for this shot on the B300 (64-wide x-pair
# tiles, 32 rows, 64-plane segments, one CTA per SM, whole segments).
BENCH_TILE = dict(tile_x=64, tile_y=32, zblock=64, ctas_per_sm=1, aligned=1, skip_c=0)
TILES_256 = {
    "default": None,
    "bench_xp": BENCH_TILE,
    "bench_xp_skip_c": dict(BENCH_TILE, skip_c=1),
    "autotuned": "autotune",
}


@pytest.fixture(scope="module")
def shot256():
    p = fdsynth.acoustic_problem(n=256, ndim=3, so=8, nbl=40, nt=500, nrec=256, seed=0)
    ou, _, orec = oracle.acoustic(p["m"], p["dt"], p["spacing"], 8, 500, damp=p["damp"],
                                  src_coords=p["src_coords"], wavelet=p["wavelet"],
                                  rec_coords=p["rec_coords"])
    assert np.abs(orec).max() > 0
    return p, ou, orec


@pytest.mark.parametrize("name", list(TILES_256))
def test_full_shot_256_so8_500_steps(shot256, name):
    from paper_1906_10811_b300 import Solver
    p, ou, orec = shot256
    tile = TILES_256[name]
    with Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic") as s:
        s.set_model(p["m"], p["damp"])
        s.set_sources(p["src_coords"], p["wavelet"])
        s.set_receivers(p["rec_coords"])
        if tile == "autotune":
            s.autotune(reps=3)
        elif tile is not None:
            s.set_tile_config(**tile)
        used = s.tile_config
        s.run(500)
        u, rec = s.read()
        kname = s.kernel_name
        skipped = s.skipped_c_planes()
    if isinstance(tile, dict):
        for k, v in tile.items():
            assert used[k] == v, (k, used)
    assert kname == ("stencil3d_xp_acoustic" if used["tile_x"] == 64 else
                     "stencil3d_tma_acoustic"), (kname, used)
    if used["skip_c"]:
        assert skipped[0] > 0, skipped        # undamped tile-planes really skip C
    ew, er = rel_l2(u, ou), rel_l2(rec, orec)
    assert ew <= TOL_WAVE, (used, ew)
    assert er <= TOL_WAVE, (used, er)


def _model_512(so):
    n = 512
    rng = np.random.default_rng(so)
    v = rng.uniform(1.5, 4.5, (n, n, n)).astype(np.float32)
    m = fdsynth.slowness_squared(v)
    damp = fdsynth.damping_profile((n,) * 3, (10.0,) * 3, v, nbl=40)
    dt = fdsynth.cfl_dt(v, 10.0, 3)
    u = fdsynth.random_field((n,) * 3, seed=so + 1)
    up = fdsynth.random_field((n,) * 3, seed=so + 2)
    return m, damp, dt, u, up


def _sample_points(n, R, rng):
    pts = [tuple(rng.integers(0, n, 3)) for _ in range(3000)]
    for c in range(8):
        pts.append(tuple((n - 1) * ((c >> k) & 1) for k in range(3)))
    for _ in range(300):  # seams of 32-wide tiles in x and y, z anywhere
        z = int(rng.integers(0, n))
        x = 32 * int(rng.integers(0, n // 32)) + int(rng.choice([0, 31]))
        y = 16 * int(rng.integers(0, n // 16)) + int(rng.choice([0, 15]))
        pts.append((z, y, x))
    for z in (0, 1, R - 1, R, n // 2 - 1, n // 2, n - R - 1, n - 1):
        pts.append((z, int(rng.integers(0, n)), int(rng.integers(0, n))))
    return pts


def _window(a, p, R, fill):
    n = a.shape[0]
    w = np.full((2 * R + 1,) * 3, fill, dtype=np.float64)
    lo = [max(0, c - R) for c in p]
    hi = [min(n, c + R + 1) for c in p]
    w[tuple(slice(l - (c - R), h - (c - R)) for l, h, c in zip(lo, hi, p))] = \
        a[tuple(slice(l, h) for l, h in zip(lo, hi))]
    return w


@pytest.mark.parametrize("so", (4, 8, 12, 16))
def test_one_step_512_sampled(so):
    from paper_1906_10811_b300 import Solver
    R = so // 2
    m, damp, dt, u, up = _model_512(so)
    with Solver((512,) * 3, (10.0,) * 3, so, dt, "acoustic") as s:
        s.set_model(m, damp)
        s.set_field(u, up)
        s.run(1)
        g, _ = s.read()
    rng = np.random.default_rng(100 + so)
    got, ref = [], []
    for p in _sample_points(512, R, rng):
        mw = np.ones((2 * R + 1,) * 3)
        dw = np.zeros((2 * R + 1,) * 3)
        mw[R, R, R] = m[p]
        dw[R, R, R] = damp[p]
        o, _, _ = oracle.acoustic(mw, dt, (10.0,) * 3, so, 1, damp=dw,
                                  u_cur=_window(u, p, R, 0.0), u_prev=_window(up, p, R, 0.0))
        got.append(g[p])
        ref.append(o[R, R, R])
    got, ref = np.array(got, np.float64), np.array(ref)
    assert rel_l2(got, ref) <= 1e-5
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("so", (8, 16))
def test_twenty_steps_512_whole_grid(so):
    """The default tile and the autotuned one (the bench's sweep configuration):
    bitwise the same, and within the tolerance of the oracle on the whole grid."""
    from paper_1906_10811_b300 import Solver
    m, damp, dt, u, up = _model_512(so)
    runs = []
    for tune in (False, True):
        with Solver((512,) * 3, (10.0,) * 3, so, dt, "acoustic") as s:
            s.set_model(m, damp)
            if tune:
                s.autotune(reps=2)
            s.set_field(u, up)
            s.run(20)
            g, _ = s.read()
            runs.append((g, s.read_prev(), s.tile_config))
    (g, gp, _), (gt, gpt, used) = runs
    assert np.array_equal(g, gt) and np.array_equal(gp, gpt), used
    ou, oup, _ = oracle.acoustic(m, dt, (10.0,) * 3, so, 20, damp=damp, u_cur=u, u_prev=up)
    assert rel_l2(g, ou) <= TOL_WAVE
    assert rel_l2(gp, oup) <= TOL_WAVE


# ---------------------------------------------------------------------------
# 512³ in the configurations the bench's sweep runs: the autotuner picks the tile
# (on the B300: the x-pair kernel's work queue, 24-row tiles of 12 consumer warps
# at so 12 and 16), then one step is checked on sampled points.

@pytest.mark.parametrize("so", (4, 8, 12, 16))
def test_one_step_512_sampled_tuned_tile(so):
    from paper_1906_10811_b300 import Solver
    R = so // 2
    m, damp, dt, u, up = _model_512(so)
    with Solver((512,) * 3, (10.0,) * 3, so, dt, "acoustic") as s:
        s.set_model(m, damp)
        s.autotune(reps=2)
        used = s.tile_config
        s.set_field(u, up)
        s.run(1)
        g, _ = s.read()
    rng = np.random.default_rng(200 + so)
    got, ref = [], []
    for p in _sample_points(512, R, rng):
        mw = np.ones((2 * R + 1,) * 3)
        dw = np.zeros((2 * R + 1,) * 3)
        mw[R, R, R] = m[p]
        dw[R, R, R] = damp[p]
        o, _, _ = oracle.acoustic(mw, dt, (10.0,) * 3, so, 1, damp=dw,
                                  u_cur=_window(u, p, R, 0.0), u_prev=_window(up, p, R, 0.0))
        got.append(g[p])
        ref.append(o[R, R, R])
    got, ref = np.array(got, np.float64), np.array(ref)
    assert rel_l2(got, ref) <= 1e-5, used
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), used


@pytest.mark.parametrize("so", (4, 8, 16))
def test_diffusion_one_step_512_sampled_tuned_tile(so):
    """The 512³ diffusion sweep's step (ν dt/h² = 0.05) from a random field, tile
    autotuned: sampled interior points against the oracle on (2R+1)³ windows, boundary
    nodes unchanged."""
    from paper_1906_10811_b300 import Solver
    R, n = so // 2, 512
    h = 1.0 / (n - 1)
    nu, dt = 0.5, 0.05 * h * h / 0.5
    u = fdsynth.random_field((n,) * 3, seed=300 + so)
    with Solver((n,) * 3, (h,) * 3, so, dt, "diffusion", nu=nu) as s:
        s.autotune(reps=2)
        used = s.tile_config
        s.set_field(u)
        s.run(1)
        g, _ = s.read()
    rng = np.random.default_rng(400 + so)
    got, ref = [], []
    for p in _sample_points(n, R, rng):
        if min(p) == 0 or max(p) == n - 1:   # boundary node: held
            assert g[p] == u[p], (p, used)
            continue
        o = oracle.diffusion(_window(u, p, R, 0.0), (h,) * 3, so, nu, dt, 1)
        got.append(g[p])
        ref.append(o[R, R, R])
    got, ref = np.array(got, np.float64), np.array(ref)
    assert rel_l2(got, ref) <= 1e-5, used
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), used
