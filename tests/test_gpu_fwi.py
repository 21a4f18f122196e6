"""FWI on the device: the adjoint solver passes the dot-product test against the
forward modelling operator, the gradient matches the FP64 oracle's
adjoint-state gradient (itself pinned by finite differences), passes a Taylor
test, does not depend on the checkpoint interval, and comes back through
torch.autograd."""

import numpy as np
import pytest

import fdsynth
from helpers import rel_l2
from oracle import fwi as ofwi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _shot(shape=(30, 34, 38), nt=120, seed=0, nrec=16, nsrc=1):
    nd = len(shape)
    p = fdsynth.acoustic_problem(n=shape, ndim=nd, so=8, nbl=5, nt=nt, nrec=nrec, seed=seed, f0=0.03)
    if nsrc > 1:
        p["src_coords"] = fdsynth.random_points(shape, p["spacing"], nsrc, seed=seed + 5, margin=7.0)
        p["wavelet"] = np.repeat(p["wavelet"], nsrc, axis=1) * np.linspace(0.5, 1.5, nsrc,
                                                                            dtype=np.float32)
    return p


def _true_model(p):
    """The observed data come from the model with a smooth positive anomaly."""
    shape = p["shape"]
    g = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    r2 = sum((x - (n - 1) / 2.0) ** 2 for x, n in zip(g, shape))
    return (p["m"] * (1.0 + 0.08 * np.exp(-r2 / 30.0))).astype(np.float32)


def test_adjoint_dot_product():
    """<F x, y> = <x, Fᵀ y> for F: source wavelets -> receiver traces."""
    import torch
    from paper_1906_10811_b300 import Solver
    p = _shot(nsrc=3)
    nt = p["nt"]
    rng = np.random.default_rng(1)
    x = rng.standard_normal((nt, 3)).astype(np.float32)
    y = rng.standard_normal((nt + 1, len(p["rec_coords"]))).astype(np.float32)
    with Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic") as s:
        s.set_model(p["m"], p["damp"])
        s.set_sources(p["src_coords"], x)
        s.set_receivers(p["rec_coords"])
        s.run(nt)
        _, fx = s.read(field=False)
    with Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic") as a:
        a.set_model(p["m"], p["damp"])
        a.set_sources(p["rec_coords"], np.ascontiguousarray(y[1:][::-1]))
        a.set_receivers(p["src_coords"])
        a.run(nt)
        _, sa = a.read(field=False)
    fty = sa[nt - np.arange(nt)]                       # s_n = rec_a[nt - n]
    lhs = float(np.sum(fx.astype(np.float64) * y))
    rhs = float(np.sum(x.astype(np.float64) * fty))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


def test_gradient_matches_oracle():
    from paper_1906_10811_b300 import fwi
    p = _shot()
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    J, g = fwi.gradient(p, d_obs)
    Jo, go = ofwi.gradient(p["m"], p["damp"], p["dt"], p["spacing"], 8, p["nt"], p["src_coords"],
                           p["wavelet"], p["rec_coords"], d_obs)
    assert abs(J - Jo) <= 1e-4 * Jo
    assert rel_l2(g.cpu().numpy(), go) <= 1e-4


def test_checkpoint_interval_does_not_change_the_gradient():
    from paper_1906_10811_b300 import fwi
    p = _shot(shape=(26, 24, 29), nt=60)
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    ref = fwi.gradient(p, d_obs, k=60)[1].cpu().numpy()
    for k in (1, 7, 25):
        assert np.array_equal(fwi.gradient(p, d_obs, k=k)[1].cpu().numpy(), ref)
    assert fwi.choose_checkpoint_interval(1000, 100, 100 * 1004) == 1000   # nt + 2 + 2 levels
    assert fwi.choose_checkpoint_interval(1000, 100, 100 * 100) < 100


def test_taylor_second_order():
    """J(m + h δm) − J(m) − h <g, δm> shrinks by about 4 when h halves."""
    from paper_1906_10811_b300 import fwi
    p = _shot(shape=(28, 26, 30), nt=100)
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    J0, g = fwi.gradient(p, d_obs)
    g = g.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(4)
    dm = (rng.standard_normal(p["shape"]) * p["m"] * 0.02).astype(np.float64)
    rem = []
    for h in (1.0, 0.5, 0.25):
        mh = (p["m"] + h * dm).astype(np.float32)
        r = fwi.forward_traces(p, mh).cpu().numpy().astype(np.float64) - d_obs
        Jh = 0.5 * np.sum(r * r)
        rem.append(abs(Jh - J0 - h * np.sum(g * dm)))
    first = [abs(0.5 * np.sum((fwi.forward_traces(p, (p["m"] + h * dm).astype(np.float32)).cpu().numpy() - d_obs) ** 2) - J0)
             for h in (1.0, 0.5, 0.25)]
    for a, b in zip(rem, rem[1:]):
        assert 3.0 < a / b < 5.0, rem
    assert rem[-1] < 0.1 * first[-1]


def test_autograd_returns_the_gradient():
    import torch
    from paper_1906_10811_b300 import fwi
    p = _shot(shape=(22, 24, 26), nt=50)
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    m = torch.tensor(p["m"], device="cuda", requires_grad=True)
    J = fwi.FWIObjective.apply(m, p, d_obs, None)
    J.backward()
    _, g = fwi.gradient(p, d_obs)
    assert torch.equal(m.grad, g)
    assert abs(float(J) - fwi.gradient(p, d_obs)[0]) <= 1e-12 * float(J)


def test_checkpoint_interval_tuner_times_candidates_and_keeps_the_gradient():
    from paper_1906_10811_b300 import fwi
    p = _shot(shape=(24, 22, 27), nt=48)
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    k, rows = fwi.tune_checkpoint_interval(p, d_obs, candidates=[4, 12, 48])
    assert [r[0] for r in rows] == [4, 12, 48]
    assert k in (4, 12, 48)
    assert all(r[1] > 0 for r in rows)
    fastest = min(r[1] for r in rows)
    chosen = [r for r in rows if r[0] == k][0]
    assert chosen[1] <= 1.03 * fastest
    ref = fwi.gradient(p, d_obs, k=48)[1]
    import torch
    assert torch.equal(fwi.gradient(p, d_obs, k=k)[1], ref)
    st = {}
    fwi.gradient(p, d_obs, k=k, stats=st)
    assert st["k"] == k and st["launches_forward"] > 0 and st["launches_adjoint"] > 0
    import math
    fb = st["checkpoint_bytes"] // (2 * math.ceil(48 / k))       # bytes of one padded level
    levels = k + 1 if st["fused"] else k + 2                      # d2 levels + padded gradient
    assert st["block_bytes"] == levels * fb
    assert st["checkpoint_bytes"] + st["block_bytes"] <= fwi.checkpoint_memory(48, k, fb)


def test_fused_backward_sweep_is_bitwise_the_separate_kernels():
    """fd_step_fwi computes the second time difference in the recompute's epilogue and
    the imaging condition in the adjoint's: the same arithmetic as fd_snapshot +
    fd_imaging, so the same gradient bit for bit, for several k."""
    import torch
    from paper_1906_10811_b300 import fwi
    p = _shot(shape=(29, 33, 40), nt=70)
    d_obs = fwi.forward_traces(p, _true_model(p)).cpu().numpy()
    for k in (9, 70):
        st = {}
        Ja, ga = fwi.gradient(p, d_obs, k=k, fused=False)
        Jb, gb = fwi.gradient(p, d_obs, k=k, fused=True, stats=st)
        assert st["fused"]
        assert Ja == Jb
        assert torch.equal(ga, gb)


def test_fused_step_is_refused_where_it_does_not_apply():
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300 import binding as B
    import torch
    p = _shot(shape=(40, 44), nt=10)
    with Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", device=True) as s:
        s.set_model(torch.as_tensor(p["m"], device="cuda"))
        buf = torch.empty(B.fd_field_elems(s.ctx), device="cuda")
        with pytest.raises(B.FdError) as e:
            B.fd_step_fwi(s.ctx, d2_out=buf)
        assert e.value.status == B.FD_EUNSUPPORTED
    q = _shot(shape=(20, 22, 24), nt=10)
    with Solver(q["shape"], q["spacing"], 8, q["dt"], "acoustic", device=True) as s:
        s.set_model(torch.as_tensor(q["m"], device="cuda"))
        buf = torch.empty(B.fd_field_elems(s.ctx), device="cuda")
        with pytest.raises(B.FdError) as e:
            B.fd_step_fwi(s.ctx, img_g=buf)
        assert e.value.status == B.FD_EINVAL
        B.fd_step_fwi(s.ctx, d2_out=buf)
        assert s.steps == 1


@pytest.mark.parametrize("cfg", [dict(tile_y=16), dict(tile_y=32, aligned=1),
                                 dict(tile_y=32, zblock=9, ctas_per_sm=1, aligned=0)])
def test_fused_epilogues_match_snapshots_and_imaging_for_every_tile(cfg):
    """fd_step_fwi's d2 equals the second difference of snapshots, and its imaging
    accumulation equals fd_imaging, bit for bit, whatever the tile configuration."""
    import torch
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300 import binding as B
    p = _shot(shape=(26, 30, 37), nt=40)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    # one stream for the library calls and the torch ops between them (the binding
    # calls below do not order a private solver stream with torch's)
    work = torch.cuda.Stream()
    with torch.cuda.stream(work), \
            Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", device=True) as f, \
            Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", device=True) as a:
        for s in (f, a):
            s.set_model(dev(p["m"]), dev(p["damp"]))
            s.set_tile_config(**cfg)
        f.set_sources(dev(p["src_coords"]), dev(p["wavelet"]))
        a.set_sources(dev(p["rec_coords"][:3]), dev(np.ones((40, 3), np.float32)))
        n = B.fd_field_elems(f.ctx)
        f.run(7)
        a.run(7)
        cur, prev = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        nxt, d2 = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        g_pad = torch.zeros(n, device="cuda")
        for _ in range(5):
            B.fd_snapshot(f.ctx, cur, prev)
            B.fd_step_fwi(f.ctx, d2_out=d2)
            B.fd_snapshot(f.ctx, nxt)
            want = torch.empty(p["shape"], device="cuda")
            got = torch.empty(p["shape"], device="cuda")
            B.fd_field_to_dense(f.ctx, (nxt - cur) - (cur - prev), want)
            B.fd_field_to_dense(f.ctx, d2, got)
            assert torch.equal(got, want)
            # the fused imaging against fd_imaging after the same adjoint step
            gd = torch.zeros(p["shape"], device="cuda")
            g_pad.zero_()
            B.fd_step_fwi(a.ctx, img_g=g_pad, img_d2=d2, scale=-0.37)
            B.fd_imaging(a.ctx, gd, nxt, cur, prev, -0.37)
            gfused = torch.empty(p["shape"], device="cuda")
            B.fd_field_to_dense(a.ctx, g_pad, gfused)
            assert torch.equal(gfused, gd)
        torch.cuda.synchronize()


@pytest.mark.parametrize("reverse", (False, True))
def test_run_fwi_sequence_is_bitwise_the_single_steps(reverse):
    """fd_run_fwi (graph-replayed chunks; 70 steps = a 64-step chunk and a 6-step one)
    writes and reads the same rows as fd_step_fwi called step by step."""
    import torch
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300 import binding as B
    p = _shot(shape=(26, 30, 41), nt=160)        # wavelet long enough for 10 + 2 × 70 steps
    nt = 70
    out = []
    # one stream for the library calls and the torch ops that fill their buffers (the
    # binding calls below do not order a private solver stream with torch's)
    work = torch.cuda.Stream()
    for seq in (False, True):
        with torch.cuda.stream(work), \
                Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", device=True) as s:
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            s.set_model(dev(p["m"]), dev(p["damp"]))
            s.set_sources(dev(p["src_coords"]), dev(p["wavelet"]))
            s.run(10)
            elems = B.fd_field_elems(s.ctx)
            d2 = torch.full((nt, elems), float("nan"), device="cuda")
            g = torch.zeros(elems, device="cuda")
            src = torch.randn((nt, elems), device="cuda",
                              generator=torch.Generator("cuda").manual_seed(3))
            if seq:
                B.fd_run_fwi(s.ctx, nt, d2_base=d2, stride=elems, reverse=reverse)
                B.fd_run_fwi(s.ctx, nt, img_d2_base=src, stride=elems, reverse=reverse,
                             img_g=g, scale=-0.5)
            else:
                for i in range(nt):
                    r = nt - 1 - i if reverse else i
                    B.fd_step_fwi(s.ctx, d2_out=d2[r])
                for i in range(nt):
                    r = nt - 1 - i if reverse else i
                    B.fd_step_fwi(s.ctx, img_g=g, img_d2=src[r], scale=-0.5)
            u, _ = s.read()
            out.append((u.cpu().numpy(), d2.cpu().numpy(), g.cpu().numpy()))
    for a, b in zip(*out):
        assert np.array_equal(a, b, equal_nan=True)


def test_residual_misfit_and_adjoint_wavelet():
    """fd_residual: the residual of the recorded traces, time reversed into the adjoint
    wavelet, and J = ½||r||² accumulated in double."""
    import torch
    from paper_1906_10811_b300 import Solver
    from paper_1906_10811_b300 import binding as B
    p = _shot(shape=(24, 28, 30), nt=77, nrec=37)
    rng = np.random.default_rng(8)
    work = torch.cuda.Stream()  # the library and the torch ops on one stream (as above)
    with torch.cuda.stream(work), \
            Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic", device=True) as s:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        s.set_model(dev(p["m"]), dev(p["damp"]))
        s.set_sources(dev(p["src_coords"]), dev(p["wavelet"]))
        s.set_receivers(dev(p["rec_coords"]))
        with pytest.raises(B.FdError) as e:
            B.fd_residual(s.ctx, torch.zeros((1, 37), device="cuda"))   # nothing recorded yet
        assert e.value.status == B.FD_ESTATE
        s.run(77)
        _, rec = s.read(field=False)
        d_obs = dev(rng.standard_normal((78, 37)).astype(np.float32) * float(rec.abs().max()))
        wav = torch.full((77, 37), float("nan"), device="cuda")
        J = B.fd_residual(s.ctx, d_obs, wav)
        J2 = B.fd_residual(s.ctx, d_obs)                  # no wavelet: J only, same value
        r = (rec - d_obs).cpu().numpy()                   # float32 subtraction, as recorded
        wav_h = wav.cpu().numpy()
    assert np.array_equal(wav_h, r[1:][::-1])
    Jref = 0.5 * float(np.sum(r.astype(np.float64) ** 2))
    assert J == J2
    assert abs(J - Jref) <= 1e-12 * Jref
