"""Parity at full benchmark sizes, in the launch configuration bench.py times.

* 256³ so 8 shot (damping layer 40, layered model, Ricker source at the centre,
  256 receivers, 500 steps) against the FP64 oracle on the whole grid: the
  wavefield and the traces within 1e-4 relative L2.
* 512³ at so 4/8/12/16: one step from random fields, checked on sampled points
  (random, grid corners, tile and z-block seams) against the oracle evaluated
  point by point on (2R+1)³ windows; and 20 steps at so 8 and 16 against the
  oracle on the whole grid.
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


def test_full_shot_256_so8_500_steps():
    from paper_1906_10811_b300 import Solver
    p = fdsynth.acoustic_problem(n=256, ndim=3, so=8, nbl=40, nt=500, nrec=256, seed=0)
    with Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic") as s:
        s.set_model(p["m"], p["damp"])
        s.set_sources(p["src_coords"], p["wavelet"])
        s.set_receivers(p["rec_coords"])
        s.run(500)
        u, rec = s.read()
        assert s.kernel_name == "stencil3d_tma_acoustic"
    ou, _, orec = oracle.acoustic(p["m"], p["dt"], p["spacing"], 8, 500, damp=p["damp"],
                                  src_coords=p["src_coords"], wavelet=p["wavelet"],
                                  rec_coords=p["rec_coords"])
    assert np.abs(orec).max() > 0
    assert rel_l2(u, ou) <= TOL_WAVE
    assert rel_l2(rec, orec) <= TOL_WAVE


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
    from paper_1906_10811_b300 import Solver
    m, damp, dt, u, up = _model_512(so)
    with Solver((512,) * 3, (10.0,) * 3, so, dt, "acoustic") as s:
        s.set_model(m, damp)
        s.set_field(u, up)
        s.run(20)
        g, _ = s.read()
        gp = s.read_prev()
    ou, oup, _ = oracle.acoustic(m, dt, (10.0,) * 3, so, 20, damp=damp, u_cur=u, u_prev=up)
    assert rel_l2(g, ou) <= TOL_WAVE
    assert rel_l2(gp, oup) <= TOL_WAVE
