"""GPU parity through the C ABI against the FP64 oracle, on sizes the oracle
finishes in seconds that still span several tiles and ragged edges.

Tolerances (the accuracy targets of the path, FP32 GPU vs FP64 oracle, relative
L2 over all values): diffusion 1e-5, acoustic wavefield and traces 1e-4.
Where two GPU runs must agree exactly (graphs vs eager launches, chunked runs,
host vs device pointers, resume from a checkpoint), the comparison is bitwise:
with one source no two atomic additions meet, so the arithmetic is identical.
"""

import math

import numpy as np
import pytest

import fdsynth
from helpers import gpu_acoustic, oracle_acoustic, rel_l2, small_problem
from oracle import core as oracle

pytestmark = pytest.mark.gpu

TOL_DIFF = 1e-5
TOL_WAVE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


# ----------------------------------------------------------------------------
# Diffusion (thesis §5.1.2)
# ----------------------------------------------------------------------------
def test_diffusion_benchmark_problem():
    """128² nodes, ν = 0.5, so 2, ν dt/h² = 0.2, 100 steps."""
    from paper_1906_10811_b300 import Solver
    p = fdsynth.diffusion_problem(128)
    with Solver((128, 128), p["spacing"], 2, p["dt"], "diffusion", nu=0.5) as s:
        s.set_field(p["u0"])
        s.run(100)
        u, _ = s.read()
    ref = oracle.diffusion(p["u0"], p["spacing"], 2, 0.5, p["dt"], 100)
    assert rel_l2(u, ref) <= TOL_DIFF
    h = p["spacing"][0]
    g = 1 - 4 * 0.2 * 2 * math.sin(math.pi * h / 2) ** 2
    assert rel_l2(u, g ** 100 * p["u0"].astype(np.float64)) <= TOL_DIFF
    assert np.all(u[0] == 0) and np.all(u[:, -1] == 0)


@pytest.mark.parametrize("so", (2, 4, 8, 12, 16))
@pytest.mark.parametrize("shape", [(37, 45), (3, 70), (19, 23, 41), (3, 5, 4), (9, 34, 33)])
def test_diffusion_parity(so, shape):
    from paper_1906_10811_b300 import Solver, fd_stability_symbol
    nd = len(shape)
    rng = np.random.default_rng(so + 10 * nd)
    u0 = fdsynth.random_field(shape, seed=so)
    h = tuple(rng.uniform(0.5, 1.5, nd))
    lam = sum(fd_stability_symbol(so) / hd ** 2 for hd in h)
    nu = 0.7
    dt = fdsynth.f32(0.9 * 2 / (nu * lam))
    with Solver(shape, h, so, dt, "diffusion", nu=nu) as s:
        s.set_field(u0)
        s.run(25)
        u, _ = s.read()
    ref = oracle.diffusion(u0, h, so, nu, dt, 25)
    assert rel_l2(u, ref) <= TOL_DIFF


@pytest.mark.parametrize("so", (2, 4, 8, 12, 16))
@pytest.mark.parametrize("kernel", ("plain", "auto"))
@pytest.mark.parametrize("shape", [(30, 41), (17, 23, 41), (9, 34, 33)])
def test_diffusion_odd_reflection_parity(so, kernel, shape):
    """Odd-reflection boundary: random data against the oracle's odd mode."""
    from paper_1906_10811_b300 import Solver, fd_stability_symbol
    nd = len(shape)
    u0 = fdsynth.random_field(shape, seed=so + 1)
    for d in range(nd):                       # boundary nodes hold 0
        for i in (0, shape[d] - 1):
            sl = [slice(None)] * nd
            sl[d] = i
            u0[tuple(sl)] = 0.0
    h = (0.8,) * nd
    lam = sum(fd_stability_symbol(so) / hd ** 2 for hd in h)
    nu = 0.6
    dt = fdsynth.f32(0.9 * 2 / (nu * lam))
    with Solver(shape, h, so, dt, "diffusion", nu=nu, kernel=kernel, boundary="odd") as s:
        s.set_field(u0)
        s.run(30)
        u, _ = s.read()
    ref = oracle.diffusion(u0, h, so, nu, dt, 30, boundary="odd")
    assert rel_l2(u, ref) <= TOL_DIFF
    zero = oracle.diffusion(u0, h, so, nu, dt, 30)
    if so > 2:
        assert rel_l2(u, zero) > 10 * TOL_DIFF      # the mode really changed the result


@pytest.mark.parametrize("so", (4, 8, 16))
def test_diffusion_odd_reflection_sine_mode_closed_form(so):
    """3-D sine mode under the odd-reflection boundary decays by the exact discrete
    factor 1 + ν dt Σ_d (w_0 + 2 Σ_j w_j cos(j π h)) / h² at every order."""
    from paper_1906_10811_b300 import Solver, fd_weights
    n = 48
    p = fdsynth.diffusion_problem(n, ndim=3, courant=0.05)
    h = p["spacing"][0]
    w = fd_weights(so)
    lam = (w[0] + 2 * sum(w[j] * math.cos(j * math.pi * h) for j in range(1, so // 2 + 1))) / h ** 2
    g = 1 + 0.5 * p["dt"] * 3 * lam
    with Solver((n,) * 3, p["spacing"], so, p["dt"], "diffusion", nu=0.5, boundary="odd") as s:
        s.set_field(p["u0"])
        s.run(60)
        u, _ = s.read()
    assert rel_l2(u, g ** 60 * p["u0"].astype(np.float64)) <= TOL_DIFF


def test_odd_reflection_is_rejected_where_it_does_not_apply():
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300.binding import FD_EINVAL, FD_EUNSUPPORTED, FdError
    with pytest.raises(FdError) as e:
        Solver((20, 20, 20), (10.0,) * 3, 8, 0.1, "acoustic", boundary="odd")
    assert e.value.status == FD_EUNSUPPORTED
    with pytest.raises(FdError) as e:
        Solver((20, 4), (1.0, 1.0), 8, 0.01, "diffusion", boundary="odd")
    assert e.value.status == FD_EINVAL


def test_diffusion_boundary_held_and_plain_vs_auto():
    from paper_1906_10811_b300 import Solver
    shape = (21, 18, 40)
    u0 = fdsynth.random_field(shape, seed=3)
    outs = []
    for kernel in ("plain", "auto"):
        with Solver(shape, (1.0,) * 3, 8, 0.05, "diffusion", nu=0.5, kernel=kernel) as s:
            s.set_field(u0)
            s.run(13)
            outs.append(s.read()[0])
    ref = oracle.diffusion(u0, (1.0,) * 3, 8, 0.5, 0.05, 13)
    for u in outs:
        assert rel_l2(u, ref) <= TOL_DIFF
        for ax in range(3):
            for i in (0, shape[ax] - 1):
                assert np.array_equal(np.take(u, i, axis=ax), np.take(u0, i, axis=ax))


# ----------------------------------------------------------------------------
# Acoustic (the seismic operator of thesis §6.2.1)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("so", (2, 4, 6, 8, 10, 12, 14, 16))
@pytest.mark.parametrize("shape", [(23, 29, 37), (40, 33, 70)])
def test_acoustic_parity_3d(so, shape):
    p = small_problem(shape, so, nt=90)
    g = gpu_acoustic(p, 90)
    o = oracle_acoustic(p, 90)
    assert rel_l2(g["u"], o["u"]) <= TOL_WAVE
    assert rel_l2(g["u_prev"], o["u_prev"]) <= TOL_WAVE
    assert rel_l2(g["rec"], o["rec"]) <= TOL_WAVE
    assert np.abs(o["rec"]).max() > 0


@pytest.mark.parametrize("so", (4, 8, 14))
def test_acoustic_parity_3d_anisotropic_spacing(so):
    """Unequal spacing per axis takes the per-axis difference form of the kernel."""
    shape, h = (27, 35, 44), (9.0, 12.0, 10.5)
    p = small_problem(shape, so, nt=80)
    v = p["vel"]
    p["spacing"] = h
    p["damp"] = fdsynth.damping_profile(shape, h, v, nbl=6)
    p["dt"] = fdsynth.cfl_dt(v, min(h), 3)
    p["src_coords"] = fdsynth.centre(shape, h).reshape(1, 3)
    p["rec_coords"] = fdsynth.receiver_line(shape, h, 12, 6)
    p["wavelet"] = fdsynth.ricker(80, p["dt"], 0.03).reshape(-1, 1)
    g = gpu_acoustic(p, 80)
    o = oracle_acoustic(p, 80)
    assert rel_l2(g["u"], o["u"]) <= TOL_WAVE
    assert rel_l2(g["rec"], o["rec"]) <= TOL_WAVE


@pytest.mark.parametrize("so", (2, 8, 16))
@pytest.mark.parametrize("shape", [(61, 53), (17, 130)])
def test_acoustic_parity_2d(so, shape):
    p = small_problem(shape, so, nt=150)
    g = gpu_acoustic(p, 150)
    o = oracle_acoustic(p, 150)
    assert rel_l2(g["u"], o["u"]) <= TOL_WAVE
    assert rel_l2(g["rec"], o["rec"]) <= TOL_WAVE


XP_TILES = {"xp16": dict(tile_x=64, tile_y=16), "xp32_aligned": dict(tile_x=64, tile_y=32, aligned=1,
                                                                       zblock=7)}


@pytest.mark.parametrize("kernel,shape", [("plain", (26, 31, 35)), ("auto", (26, 31, 35)),
                                          ("xp16", (26, 31, 35)), ("xp16", (21, 40, 131)),
                                          ("xp32_aligned", (21, 40, 131))])
def test_acoustic_kernels_many_sources_and_receivers(kernel, shape):
    """Random sources (two sharing a node) and receivers, including points on
    the grid boundary; enough of them to take the multi-block sparse path.  The
    x-pair tiles (a lane per two adjacent x points) also get sources on both
    points of one lane's pair, on several planes, and x extents of one tile and
    of two full tiles plus a ragged one."""
    so, nt = 8, 60
    p = small_problem(shape, so, nt)
    pts = fdsynth.random_points(shape, p["spacing"], 300, seed=5)
    pts[1] = pts[0]
    ext = np.array([(n - 1) * h for n, h in zip(shape, p["spacing"])], dtype=np.float32)
    pts[2] = ext
    pts[3] = 0
    h = np.array(p["spacing"], dtype=np.float32)
    for i, (z, y, x) in enumerate([(5, 7, 10), (5, 7, 11), (12, 20, 64), (12, 20, 65),
                                   (12, 21, 63), (3, 30, 34)]):
        pts[4 + i] = np.array([z, min(y, shape[1] - 1), min(x, shape[2] - 1)], np.float32) * h
    p["src_coords"] = pts
    p["wavelet"] = np.repeat(p["wavelet"], 300, axis=1) * np.linspace(0.5, 1.5, 300, dtype=np.float32)
    p["rec_coords"] = np.vstack([fdsynth.random_points(shape, p["spacing"], 400, seed=6), ext[None], np.zeros((1, 3), np.float32)])
    tile = XP_TILES.get(kernel)
    g = gpu_acoustic(p, nt, kernel="auto" if tile else kernel, tile=tile)
    if tile:
        assert g["kernel"] == "stencil3d_xp_acoustic" and g["tile"]["tile_x"] == 64, g["tile"]
        ref = gpu_acoustic(p, nt, kernel="auto")          # 32-wide: bitwise the same
        assert np.array_equal(g["u"], ref["u"]) and np.array_equal(g["rec"], ref["rec"])
    o = oracle_acoustic(p, nt)
    assert rel_l2(g["u"], o["u"]) <= TOL_WAVE
    assert rel_l2(g["rec"], o["rec"]) <= TOL_WAVE


def test_acoustic_without_damping_and_sources_matches_closed_form():
    """Homogeneous m, so 2, sine mode with u^{-1} = cos θ u^0: u^n = cos(nθ) u^0."""
    from paper_1906_10811_b300 import Solver
    shape, h, m, dt, nt = (30, 34, 38), 10.0, 0.25, 2.0, 200
    u0 = np.ones(())
    lam = 0.0
    for n, k in zip(shape, (1, 2, 3)):
        i = np.arange(n)
        u0 = np.multiply.outer(u0, np.sin(k * math.pi * (i + 1) / (n + 1)))
        lam += -4.0 * math.sin(k * math.pi / (2 * (n + 1))) ** 2
    cth = 1.0 + dt * dt * lam / (h * h) / (2 * m)
    with Solver(shape, (h,) * 3, 2, dt, "acoustic") as s:
        s.set_model(np.full(shape, m, np.float32))
        s.set_field(u0.astype(np.float32), (cth * u0).astype(np.float32))
        s.run(nt)
        u, _ = s.read()
    assert rel_l2(u, math.cos(nt * math.acos(cth)) * u0) <= TOL_WAVE


def test_graphs_eager_profile_chunks_and_device_pointers_agree_bitwise():
    p = small_problem((30, 27, 66), 8, nt=150)
    ref = gpu_acoustic(p, 150)
    variants = [
        gpu_acoustic(p, 150, graphs=False),
        gpu_acoustic(p, 150, profile=True),
        gpu_acoustic(p, 150, chunks=[1, 63, 64, 7, 15]),
        gpu_acoustic(p, 150, device=True),
        gpu_acoustic(p, 150, profile=True, graphs=False),
    ]
    for v in variants:
        assert np.array_equal(v["u"], ref["u"])
        assert np.array_equal(v["rec"], ref["rec"])
    # graph chunks timed as a whole, or every launch: 150 stencil launches either way
    for v in (variants[1], variants[4]):
        launches, ms = v["profile"]
        assert launches == 150 and ms > 0


def test_checkpoint_resume_is_bitwise():
    from paper_1906_10811_b300 import Solver
    p = small_problem((25, 30, 41), 4, nt=100)
    full = gpu_acoustic(p, 100)
    first = gpu_acoustic(p, 40)
    with Solver(p["shape"], p["spacing"], 4, p["dt"], "acoustic") as s:
        s.set_model(p["m"], p["damp"])
        s.set_field(first["u"], first["u_prev"])
        s.set_step(40)
        s.set_sources(p["src_coords"], p["wavelet"])
        s.set_receivers(p["rec_coords"])
        s.run(60)
        u, rec = s.read()
    assert np.array_equal(u, full["u"])
    assert np.array_equal(rec[41:], full["rec"][41:])
    assert np.all(rec[:40] == 0)


def test_edge_cases():
    from paper_1906_10811_b300 import Solver
    # smallest acoustic grid, one source on a corner node, receivers on nodes
    shape = (2, 2, 2)
    m = np.full(shape, 0.2, np.float32)
    wav = fdsynth.ricker(10, 1.0, 0.05).reshape(-1, 1)
    src = np.array([[10.0, 0.0, 10.0]], np.float32)
    rec = np.array([[0, 0, 0], [10, 10, 10], [5, 5, 5]], np.float32)
    with Solver(shape, (10.0,) * 3, 16, 1.0, "acoustic") as s:
        s.set_model(m)
        s.set_sources(src, wav)
        s.set_receivers(rec)
        s.run(0)
        u0, r0 = s.read()
        assert np.all(u0 == 0) and r0.shape == (1, 3)
        s.run(10)
        u, r = s.read()
    ou, _, orec = oracle.acoustic(m, 1.0, (10.0,) * 3, 16, 10, src_coords=src, wavelet=wav, rec_coords=rec)
    assert rel_l2(u, ou) <= TOL_WAVE and rel_l2(r, orec) <= TOL_WAVE
    # no receivers: read gives no traces; diffusion with one interior node
    with Solver((3, 3), (1.0, 1.0), 2, 0.1, "diffusion") as s:
        u0 = np.arange(9, dtype=np.float32).reshape(3, 3)
        s.set_field(u0)
        s.run(4)
        u, r = s.read()
        assert r is None
    assert rel_l2(u, oracle.diffusion(u0, (1.0, 1.0), 2, 0.5, 0.1, 4)) <= TOL_DIFF


def test_errors_are_reported():
    from paper_1906_10811_b300 import FdError, Solver, binding
    shape = (10, 11, 12)
    m = np.full(shape, 0.1, np.float32)         # leapfrog limit for dt: 1.43
    with Solver(shape, (10.0,) * 3, 8, 1.0, "acoustic") as s:
        with pytest.raises(FdError) as e:
            s.run(1)
        assert e.value.status == binding.FD_ESTATE
        with pytest.raises(FdError) as e:                # dt above the leapfrog limit
            s.set_model(np.full(shape, 0.01, np.float32))
        assert e.value.status == binding.FD_EINVAL
        bad = m.copy()
        bad[3, 4, 5] = 0
        with pytest.raises(FdError) as e:
            s.set_model(bad)
        assert e.value.status == binding.FD_EINVAL
        neg = np.zeros(shape, np.float32)
        neg[0, 0, 0] = -1
        with pytest.raises(FdError) as e:
            s.set_model(m, neg)
        assert e.value.status == binding.FD_EINVAL
        s.set_model(m)
        with pytest.raises(FdError) as e:                # outside the grid
            s.set_sources(np.array([[0, 0, 111.0]], np.float32), np.zeros((5, 1), np.float32))
        assert e.value.status == binding.FD_EINVAL
        s.set_sources(np.array([[50, 50, 50.0]], np.float32), np.zeros((5, 1), np.float32))
        with pytest.raises(FdError) as e:                # wavelet too short
            s.run(6)
        assert e.value.status == binding.FD_EINVAL
        s.run(5)
        assert s.steps == 5
    with Solver((8, 8), (1.0, 1.0), 2, 0.1, "diffusion") as s:
        with pytest.raises(FdError) as e:
            s.set_sources(np.array([[1.0, 1.0]], np.float32), np.zeros((5, 1), np.float32))
        assert e.value.status == binding.FD_EUNSUPPORTED


@pytest.mark.parametrize("so", (2, 8, 16))
@pytest.mark.parametrize("shape", [(61, 53), (17, 130), (100, 37), (530, 601), (1500, 90)])
def test_2d_streamed_rows_are_bitwise_the_plain_kernel(so, shape):
    """FD_KERNEL_TMA on 2-D grids runs the row-streaming kernel (warps over 64-column
    strips and row segments, rows staged with cp.async, y neighbours from registers;
    ragged strips, one or many segments); its per-point arithmetic is the plain
    kernel's, so both give the same bits, with sources and receivers (acoustic), the
    held boundary and the odd reflection (diffusion)."""
    from paper_1906_10811_b300 import Solver
    p = small_problem(shape, so, nt=90)
    streamed = gpu_acoustic(p, 90, kernel="tma")
    plain = gpu_acoustic(p, 90, kernel="plain")
    assert streamed["kernel"] == "stencil2d_stream" and plain["kernel"] == "stencil2d_plain"
    assert np.array_equal(streamed["u"], plain["u"])
    assert np.array_equal(streamed["rec"], plain["rec"])
    rng = np.random.default_rng(so)
    u0 = rng.standard_normal(shape).astype(np.float32)
    h = (1.0 / 40, 1.0 / 30)
    for boundary in ("zero", "odd"):
        if boundary == "odd" and min(shape) - 1 < so // 2:
            continue
        outs = []
        for kernel in ("tma", "plain"):
            with Solver(shape, h, so, 0.05 * min(h) ** 2, "diffusion", kernel=kernel,
                        boundary=boundary) as s:
                s.set_field(u0)
                s.run(40)
                outs.append(s.read()[0])
        assert np.array_equal(outs[0], outs[1]), boundary
        assert np.array_equal(outs[0][0], u0[0]) and np.array_equal(outs[0][:, -1], u0[:, -1])


@pytest.mark.parametrize("kernel,shape,tile", [
    ("plain", (41, 37), None), ("tma", (41, 37), None), ("plain", (23, 29, 70), None),
    ("tma", (23, 29, 70), None), ("tma", (23, 29, 131), dict(tile_x=64, tile_y=16)),
    ("tma", (23, 29, 70), dict(tile_y=16, aligned=1, zblock=7))])
@pytest.mark.parametrize("so", (2, 8, 16))
def test_diffusion_every_node_updated(kernel, shape, tile, so):
    """dirichlet_interior = 0: every node updated with zeros outside the grid (§2.1.1's
    operator without the interior subdomain), against the oracle's all-node sweep."""
    from paper_1906_10811_b300 import Solver
    rng = np.random.default_rng(so + len(shape))
    u0 = rng.standard_normal(shape).astype(np.float32)
    h = tuple(1.0 / (n + 1) for n in shape)
    dt = 0.05 * min(h) ** 2
    with Solver(shape, h, so, dt, "diffusion", kernel=kernel, dirichlet_interior=False) as s:
        if tile:
            s.set_tile_config(**tile)
        s.set_field(u0)
        s.run(30)
        u, _ = s.read()
    ref = oracle.diffusion(u0, h, so, 0.5, dt, 30, interior=False)
    assert rel_l2(u, ref) <= 1e-5
    assert np.abs(u[0] - u0[0]).max() > 0          # boundary nodes move
    held = oracle.diffusion(u0, h, so, 0.5, dt, 30)
    assert rel_l2(held, ref) > 1e-4                # the two sweeps differ measurably


@pytest.mark.parametrize("so", (2, 4))
@pytest.mark.parametrize("shape", [(61, 53), (17, 130), (530, 601), (1500, 90)])
def test_2d_diffusion_two_steps_a_launch_are_bitwise_single_steps(so, shape):
    """2-D diffusion at radius 1-2 streams pairs of steps (u^{n+2} from u^n in one
    pass, the intermediate level on a strip widened by R columns each side): bitwise
    the plain kernel's single steps, for equal and unequal spacing, the held boundary
    and every node updated, over chunks of odd lengths (a single step closes each),
    with graph replay and with eager launches."""
    from paper_1906_10811_b300 import Solver
    rng = np.random.default_rng(so * 7 + shape[0])
    u0 = rng.standard_normal(shape).astype(np.float32)
    for h in ((1.0 / 50, 1.0 / 50), (1.0 / 40, 1.0 / 30)):
        for hold in (True, False):
            outs = []
            for kernel, graphs in (("plain", True), ("tma", True), ("tma", False)):
                with Solver(shape, h, so, 0.05 * min(h) ** 2, "diffusion", kernel=kernel,
                            graphs=graphs, dirichlet_interior=hold) as s:
                    if kernel == "tma":
                        assert s.kernel_name == "stencil2d_stream2"
                    s.set_field(u0)
                    for n in (1, 3, 40, 2):
                        s.run(n)
                    assert s.steps == 46
                    outs.append(s.read()[0])
            assert np.array_equal(outs[1], outs[0]), (h, hold)
            assert np.array_equal(outs[2], outs[0]), (h, hold)
            ref = oracle.diffusion(u0, h, so, 0.5, 0.05 * min(h) ** 2, 46, interior=hold)
            assert rel_l2(outs[0], ref) <= 1e-5


@pytest.mark.parametrize("so", (2, 4))
def test_2d_two_step_stream_with_two_pairs_a_lane(so):
    """On a grid with enough 124-column strips to fill the GPU, the two-step stream
    gives each lane two pairs (a 128-column intermediate strip): bitwise the plain
    kernel's single steps, equal and unequal spacing, held and free boundary, a ragged
    last strip (12000 = 96 strips of 124 + 96 columns), odd step count."""
    from paper_1906_10811_b300 import Solver
    shape = (4000, 12000)
    rng = np.random.default_rng(11 + so)
    u0 = rng.standard_normal(shape).astype(np.float32)
    for h in ((1.0 / 50, 1.0 / 50), (1.0 / 40, 1.0 / 30)):
        for hold in (True, False):
            outs = []
            for kernel in ("plain", "tma"):
                with Solver(shape, h, so, 0.05 * min(h) ** 2, "diffusion", kernel=kernel,
                            dirichlet_interior=hold) as s:
                    if kernel == "tma":
                        assert s.kernel_name == "stencil2d_stream2"
                    s.set_field(u0)
                    s.run(5)
                    outs.append(s.read()[0])
            assert np.array_equal(outs[1], outs[0]), (h, hold)


@pytest.mark.parametrize("so,boundary", ((6, "zero"), (8, "zero"), (10, "zero"), (12, "zero"),
                                         (14, "zero"), (4, "odd")))
def test_2d_stream_with_four_points_a_lane(so, boundary):
    """At radius 2-7, where the grid has enough 128-column strips and segments of
    max(32, 2·so) rows for 64 warp streams an SM, the one-step 2-D diffusion stream
    gives each lane four adjacent points (16-byte shared-memory reads, one 16-byte
    store where all four are updated): bitwise the plain kernel, equal and unequal spacing,
    held and free boundary (zero halo; so 4 runs one step a launch with the odd
    reflection), a ragged last strip (12000 = 93 strips of 128 + 96 columns)."""
    import torch
    from paper_1906_10811_b300 import Solver
    shape = (4000, 12000)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert -(-shape[1] // 128) * (shape[0] // max(32, 2 * so)) >= 64 * sms
    rng = np.random.default_rng(23 + so)
    u0 = rng.standard_normal(shape).astype(np.float32)
    if boundary == "odd":
        u0[0, :] = u0[-1, :] = u0[:, 0] = u0[:, -1] = 0.0
    holds = (True, False) if boundary == "zero" else (True,)
    for h in ((1.0 / 50, 1.0 / 50), (1.0 / 40, 1.0 / 30)):
        for hold in holds:
            outs = []
            for kernel in ("plain", "tma"):
                with Solver(shape, h, so, 0.02 * min(h) ** 2, "diffusion", kernel=kernel,
                            dirichlet_interior=hold, boundary=boundary) as s:
                    if kernel == "tma":
                        assert s.kernel_name == "stencil2d_stream"
                    s.set_field(u0)
                    s.run(3)
                    outs.append(s.read()[0])
            assert np.array_equal(outs[1], outs[0]), (h, hold)


def test_large_2d_diffusion_streams_rows_by_default():
    """From 4 M points a 2-D diffusion context runs the row-streaming kernel unless
    asked for plain; the acoustic step keeps the plain kernel; both kernels agree."""
    from paper_1906_10811_b300 import Solver
    shape = (2100, 2003)
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(shape).astype(np.float32)
    h = (1.0 / 2099, 1.0 / 2002)
    outs = []
    for kernel, name in (("auto", "stencil2d_stream2"), ("plain", "stencil2d_plain")):
        with Solver(shape, h, 4, 0.05 * min(h) ** 2, "diffusion", kernel=kernel) as s:
            assert s.kernel_name == name
            s.set_field(u0)
            s.run(7)
            outs.append(s.read()[0])
    assert np.array_equal(outs[0], outs[1])
    with Solver(shape, (10.0, 10.0), 4, 0.1, "acoustic") as s:
        assert s.kernel_name == "stencil2d_plain"
