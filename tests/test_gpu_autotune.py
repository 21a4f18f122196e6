"""Tile configurations of the pipelined 3-D kernel and the autotuner.

A point's update is the same arithmetic whatever tile holds it, so every
configuration the kernel offers (tile height 16 or 32, CTAs per SM, z-block
height) must give bitwise the result of the default one, with sources and
receivers; the autotuner must pick one of the configurations it timed, leave
the solution untouched, and a tuned shot must still join a batch."""

import numpy as np
import pytest

from helpers import oracle_acoustic, rel_l2, small_problem

pytestmark = pytest.mark.gpu

TOL_WAVE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _acoustic(p, nt, cfg=None, tune=False, chunks=None):
    from paper_1906_10811_b300 import Solver
    s = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", kernel="tma")
    s.set_model(p["m"], p["damp"])
    s.set_sources(p["src_coords"], p["wavelet"])
    s.set_receivers(p["rec_coords"])
    if cfg is not None:
        s.set_tile_config(**cfg)
    used = s.tile_config
    for n in (chunks or [nt]):
        s.run(n)
        if tune:
            s.autotune(reps=2)
    u, rec = s.read()
    up = s.read_prev()
    s.close()
    return u, up, rec, used


def _configs(shape, so):
    """Every (tile_y, ctas_per_sm, zblock) the plan accepts for this problem."""
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300.binding import FdError
    out = []
    s = Solver(shape, (10.0,) * 3, so, 0.1, "acoustic", kernel="tma")
    for tx in (32, 64):
        for ty in (16, 24, 32):
            for cps in (1, 2, 3):
                for zb in (0, 3, 11, shape[0]):
                    for al in (0, 1, 2):
                        for sk in ((0, 1) if so <= 8 else (0,)):
                            try:
                                s.set_tile_config(tile_y=ty, ctas_per_sm=cps, zblock=zb,
                                                  aligned=al, skip_c=sk, tile_x=tx)
                            except FdError:
                                continue
                            out.append(dict(tile_y=ty, ctas_per_sm=cps, zblock=zb, aligned=al,
                                            skip_c=sk, tile_x=tx))
    s.close()
    return out


@pytest.mark.parametrize("so,shape", [(4, (37, 45, 70)), (8, (33, 50, 41)), (16, (29, 38, 66))])
def test_every_tile_configuration_is_bitwise_the_default(so, shape):
    p = small_problem(shape, so, nt=60, nrec=11)
    ref = _acoustic(p, 60)
    cfgs = _configs(shape, so)
    heights = {c["tile_y"] for c in cfgs}
    # 24 rows: 12 consumer warps of the x-pair kernel, from space order 8
    assert heights == ({16, 24, 32} if so >= 8 else {16, 32}), cfgs
    assert all(c["tile_x"] == 64 for c in cfgs if c["tile_y"] == 24)
    assert {c["tile_x"] for c in cfgs} == {32, 64}, cfgs
    for cfg in cfgs:
        u, up, rec, used = _acoustic(p, 60, cfg)
        assert used["tile_y"] == cfg["tile_y"] and used["ctas_per_sm"] == cfg["ctas_per_sm"]
        assert used["tile_x"] == cfg["tile_x"]
        assert used["aligned"] == cfg["aligned"] and used["skip_c"] == cfg["skip_c"]
        if cfg["zblock"] and cfg["aligned"] != 2:
            assert used["zblock"] == min(cfg["zblock"], shape[0])
        if cfg["aligned"] == 2:  # the queue keeps its cap as given
            assert used["zblock"] == cfg["zblock"]
        assert np.array_equal(u, ref[0]), cfg
        assert np.array_equal(up, ref[1]), cfg
        assert np.array_equal(rec, ref[2]), cfg
    o = oracle_acoustic(p, 60)
    assert rel_l2(ref[0], o["u"]) <= TOL_WAVE
    assert rel_l2(ref[2], o["rec"]) <= TOL_WAVE


@pytest.mark.parametrize("tx,ty,so", [(64, 16, 4), (64, 16, 8), (64, 16, 16), (64, 24, 16)])
def test_work_queue_with_more_items_than_ctas(tx, ty, so):
    """aligned = 2 on a grid whose queue holds more items than the grid has CTAs
    (one CTA per SM), so CTAs take several items in a row; bitwise the default tile
    and within the tolerance of the oracle; every launch of the run reuses the queue
    the previous one reset."""
    shape = (96, 100, 130)
    p = small_problem(shape, so, nt=40, nrec=21)
    ref = _acoustic(p, 40)
    cfg = dict(tile_x=tx, tile_y=ty, ctas_per_sm=1, aligned=2)
    u, up, rec, used = _acoustic(p, 40, cfg)
    assert used["aligned"] == 2 and used["tile_x"] == tx and used["tile_y"] == ty
    assert np.array_equal(u, ref[0]) and np.array_equal(up, ref[1])
    assert np.array_equal(rec, ref[2])
    o = oracle_acoustic(p, 40)
    assert rel_l2(u, o["u"]) <= TOL_WAVE
    assert rel_l2(rec, o["rec"]) <= TOL_WAVE


@pytest.mark.parametrize("so", (8, 16))
def test_diffusion_24_row_tiles_agree(so):
    """12 consumer warps (24-row x-pair tiles), static split and work queue, bitwise
    the default tile on a ragged diffusion grid."""
    from paper_1906_10811_b300 import Solver
    rng = np.random.default_rng(so)
    shape = (40, 61, 150)
    u0 = rng.standard_normal(shape).astype(np.float32)
    outs = []
    for cfg in (None, dict(tile_x=64, tile_y=24), dict(tile_x=64, tile_y=24, aligned=1),
                dict(tile_x=64, tile_y=24, aligned=2, ctas_per_sm=1)):
        s = Solver(shape, (1.0 / 60,) * 3, so, 0.05 * (1.0 / 60) ** 2, "diffusion", kernel="tma")
        if cfg:
            s.set_tile_config(**cfg)
            assert s.tile_config["tile_y"] == 24
        s.set_field(u0)
        s.run(15)
        outs.append(s.read()[0])
        s.close()
    for u in outs[1:]:
        assert np.array_equal(u, outs[0])


def test_diffusion_tile_configurations_agree():
    from paper_1906_10811_b300 import Solver
    rng = np.random.default_rng(3)
    shape = (26, 41, 67)
    u0 = rng.standard_normal(shape).astype(np.float32)
    outs = []
    for cfg in (None, dict(tile_y=16), dict(tile_y=32, zblock=5), dict(tile_y=16, ctas_per_sm=1),
                dict(aligned=1), dict(tile_y=16, zblock=9, aligned=1), dict(tile_x=64, aligned=2),
                dict(tile_x=64, tile_y=16, zblock=9, aligned=2, ctas_per_sm=1),
                dict(tile_x=64, tile_y=16, aligned=2, ctas_per_sm=1)):
        s = Solver(shape, (1.0 / 40,) * 3, 6, 0.1 * (1.0 / 40) ** 2, "diffusion", kernel="tma")
        if cfg:
            s.set_tile_config(**cfg)
        s.set_field(u0)
        s.run(25)
        outs.append(s.read()[0])
        s.close()
    for u in outs[1:]:
        assert np.array_equal(u, outs[0])


def test_autotune_picks_a_timed_configuration_and_keeps_the_solution():
    p = small_problem((48, 64, 96), 8, nt=80, nrec=16)
    ref = _acoustic(p, 80)
    # autotune between chunks of steps: the solution continues unchanged
    u, up, rec, _ = _acoustic(p, 80, tune=True, chunks=[30, 25, 25])
    assert np.array_equal(u, ref[0]) and np.array_equal(up, ref[1]) and np.array_equal(rec, ref[2])

    from paper_1906_10811_b300 import Solver
    s = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", kernel="tma")
    s.set_model(p["m"], p["damp"])
    best, tried = s.autotune(reps=3)
    assert len(tried) >= 4
    assert {t["tile_y"] for t in tried} == {16, 24, 32}
    assert {t["aligned"] for t in tried} == {0, 1, 2}
    assert all(t["tile_x"] == 64 for t in tried if t["aligned"] == 2)
    assert all(t["us_per_step"] > 0 for t in tried)
    key = lambda t: (t["tile_y"], t["zblock"], t["ctas_per_sm"], t["aligned"], t["skip_c"])
    assert {t["skip_c"] for t in tried} == {0, 1}
    assert key(best) in {key(t) for t in tried}
    assert best["us_per_step"] == min(t["us_per_step"] for t in tried)
    cur = s.tile_config
    assert key(cur) == key(best) and cur["us_per_step"] == best["us_per_step"]
    s.close()


def test_autotune_option_at_creation_uses_the_process_cache():
    from paper_1906_10811_b300 import Solver
    p = small_problem((40, 44, 52), 6, nt=10)
    a = Solver(p["shape"], p["spacing"], 6, p["dt"], "acoustic", autotune=True)
    b = Solver(p["shape"], p["spacing"], 6, p["dt"], "acoustic", autotune=True)
    ca, cb = a.tile_config, b.tile_config
    assert ca["us_per_step"] > 0
    assert ca == cb
    a.close()
    b.close()


def test_bad_tile_configurations_are_rejected_and_keep_the_current_one():
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300.binding import FD_EINVAL, FD_EUNSUPPORTED, FdError
    s = Solver((20, 24, 28), (10.0,) * 3, 8, 0.1, "acoustic", kernel="tma")
    before = s.tile_config
    for bad in (dict(tile_y=24), dict(tile_y=64), dict(zblock=-1), dict(ctas_per_sm=-2),
                dict(ctas_per_sm=64), dict(aligned=3), dict(skip_c=3), dict(tile_x=48),
                dict(tile_x=16), dict(aligned=2, tile_x=32)):
        with pytest.raises(FdError) as e:
            s.set_tile_config(**bad)
        assert e.value.status == FD_EINVAL
        assert s.tile_config == before
    s.close()
    s2 = Solver((40, 50), (10.0,) * 2, 8, 0.1, "acoustic")
    with pytest.raises(FdError) as e:
        s2.set_tile_config(tile_y=16)
    assert e.value.status == FD_EUNSUPPORTED
    s2.close()


def test_a_tuned_shot_joins_a_batch_at_the_default_tile():
    from paper_1906_10811_b300 import Batch, Solver
    p = small_problem((31, 36, 45), 8, nt=50, nrec=7)
    ref = _acoustic(p, 50)
    s = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic")
    s.set_model(p["m"], p["damp"])
    s.set_sources(p["src_coords"], p["wavelet"])
    s.set_receivers(p["rec_coords"])
    s.set_tile_config(tile_y=16, zblock=9, tile_x=64)
    s.run(20)
    b = Batch(8)
    b.add(s)
    b.run(30)
    b.remove(s)
    assert s.tile_config["tile_y"] == 32 and s.tile_config["tile_x"] == 32
    u, rec = s.read()
    up = s.read_prev()
    b.close()
    s.close()
    assert np.array_equal(u, ref[0]) and np.array_equal(up, ref[1]) and np.array_equal(rec, ref[2])


def test_fwi_autotune_times_the_sweep_kernels_and_caches():
    from paper_1906_10811_b300 import Solver
    p = small_problem((36, 40, 70), 8, nt=10)
    s = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", kernel="tma")
    s.set_model(p["m"], p["damp"])
    best, tried = s.autotune(reps=2, fwi=True)
    assert len(tried) >= 4 and all(t["us_per_step"] > 0 for t in tried)
    key = lambda t: (t["tile_y"], t["zblock"], t["ctas_per_sm"], t["aligned"], t["skip_c"])
    assert key(best) in {key(t) for t in tried}
    assert best["us_per_step"] == min(t["us_per_step"] for t in tried)
    s2 = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", kernel="tma")
    again, none = s2.autotune(fwi=True, cached=True)
    assert none == [] and key(again) == key(best)
    assert key(s2.tile_config) == key(best)
    s.close()
    s2.close()


def test_skipping_c_is_bitwise_on_a_grid_with_a_real_damping_layer():
    """160³, 40-point layer: about a fifth of the tile-planes are undamped; the step with
    their C tiles skipped is bitwise the step that reads them."""
    import fdsynth
    p = fdsynth.acoustic_problem(n=160, so=8, nbl=40, nt=40, nrec=32, seed=5)
    ref = _acoustic(p, 40, dict(tile_y=32, aligned=1, skip_c=0))
    got = _acoustic(p, 40, dict(tile_y=32, aligned=1, skip_c=1))
    assert got[3]["skip_c"] == 1
    for a, b in zip(got[:3], ref[:3]):
        assert np.array_equal(a, b)
    assert np.abs(ref[2]).max() > 0


@pytest.mark.parametrize("so,spacing,boundary", [(2, (1.0 / 40,) * 3, "zero"),
                                                 (4, (0.021, 0.025, 0.03), "zero"),
                                                 (8, (1.0 / 40,) * 3, "zero"),
                                                 (8, (1.0 / 40,) * 3, "odd"),
                                                 (12, (0.021, 0.025, 0.03), "zero"),
                                                 (16, (1.0 / 40,) * 3, "zero")])
def test_diffusion_x_pair_tiles_are_bitwise_the_default(so, spacing, boundary):
    """tile_x = 64 (a lane per pair of adjacent x points) runs the same arithmetic per
    point: bitwise the default kernel, for ragged x extents, both splits and both heights."""
    from paper_1906_10811_b300 import Solver
    rng = np.random.default_rng(so)
    shape = (23, 37, 131)                      # x: two full 64-wide tiles and 3 points
    u0 = rng.standard_normal(shape).astype(np.float32)
    dt = 0.05 * min(spacing) ** 2
    outs, used = [], []
    for cfg in (None, dict(tile_x=64, tile_y=16), dict(tile_x=64, tile_y=32),
                dict(tile_x=64, tile_y=16, aligned=1, zblock=7),
                dict(tile_x=64, tile_y=16, ctas_per_sm=1, zblock=3)):
        with Solver(shape, spacing, so, dt, "diffusion", kernel="tma", boundary=boundary) as s:
            if cfg:
                s.set_tile_config(**cfg)
            used.append(s.tile_config["tile_x"])
            s.set_field(u0)
            s.run(9)
            outs.append(s.read()[0])
    assert used == [32, 64, 64, 64, 64]
    for u in outs[1:]:
        assert np.array_equal(u, outs[0])


def test_x_pair_tiles_are_tuned():
    from paper_1906_10811_b300 import Solver
    p = small_problem((48, 64, 150), 12, 10, nrec=3)
    with Solver(p["shape"], p["spacing"], 12, p["dt"], "acoustic", kernel="tma") as s:
        s.set_model(p["m"], p["damp"])
        best, tried = s.autotune(reps=2)
        assert {t["tile_x"] for t in tried} == {32, 64}
        assert s.tile_config["tile_x"] == best["tile_x"]
        assert s.kernel_name == ("stencil3d_xp_acoustic" if best["tile_x"] == 64 else
                                 "stencil3d_tma_acoustic")
        _, tried = s.autotune(reps=2, fwi=True)   # the FWI sweep has no x-pair instance
        assert {t["tile_x"] for t in tried} == {32}
    with Solver((40, 48, 150), (1.0 / 40,) * 3, 8, 0.1 * (1.0 / 40) ** 2, "diffusion",
                kernel="tma") as s:
        s.set_field(np.ones((40, 48, 150), np.float32))
        best, tried = s.autotune(reps=2)
        assert {t["tile_x"] for t in tried} == {32, 64}
        assert s.tile_config["tile_x"] == best["tile_x"]


def _undamped_tile_planes(m, damp, dt, tx, ty):
    """Tile-planes (tx × ty tiles, z by z) where C = (m − σ)/(m + σ), σ = damp·dt/2,
    evaluated in float32 with correctly rounded operations, is 1 at every point."""
    sig = damp.astype(np.float32) * np.float32(0.5 * dt)
    mf = m.astype(np.float32)
    one = ((mf - sig) / (mf + sig)) == np.float32(1.0)
    n0, n1, n2 = m.shape
    k = 0
    for z in range(n0):
        for y0 in range(0, n1, ty):
            for x0 in range(0, n2, tx):
                k += int(np.all(one[z, y0:y0 + ty, x0:x0 + tx]))
    return k


@pytest.mark.parametrize("so", (4, 8))
def test_x_pair_tiles_skip_c_where_tile_planes_are_undamped(so):
    """64-wide tiles with the C tile really skipped: a grid wide enough that whole
    64 x 32 tile-planes lie inside the damping layer's inner region.  The flags the
    library computes are the tile-planes where damp = 0 everywhere, and the run is
    bitwise the one that reads C (x-pair and 32-wide) and within tolerance of the
    oracle."""
    import fdsynth
    from paper_1906_10811_b300 import Solver
    shape = (40, 80, 200)          # y tile rows 32..63 and x tiles 64..191 are undamped
    p = fdsynth.acoustic_problem(n=shape, ndim=3, so=so, nbl=6, nt=50, nrec=24, seed=7, f0=0.03)
    ref = _acoustic(p, 50)                                        # 32-wide default tile
    noskip = _acoustic(p, 50, dict(tile_x=64, tile_y=32, aligned=1, skip_c=0))
    cfg = dict(tile_x=64, tile_y=32, aligned=1, skip_c=1)
    got = _acoustic(p, 50, cfg)
    assert got[3]["tile_x"] == 64 and got[3]["skip_c"] == 1
    with Solver(p["shape"], p["spacing"], so, p["dt"], "acoustic", kernel="tma") as s:
        s.set_model(p["m"], p["damp"])
        s.set_tile_config(**cfg)
        flagged, total = s.skipped_c_planes()
    expect = _undamped_tile_planes(p["m"], p["damp"], p["dt"], 64, 32)
    assert total == 40 * 3 * 4
    assert flagged == expect and flagged > 0, (flagged, expect)
    for a, b, c in zip(got[:3], noskip[:3], ref[:3]):
        assert np.array_equal(a, b)
        assert np.array_equal(a, c)
    o = oracle_acoustic(p, 50)
    assert rel_l2(got[0], o["u"]) <= TOL_WAVE
    assert rel_l2(got[2], o["rec"]) <= TOL_WAVE
