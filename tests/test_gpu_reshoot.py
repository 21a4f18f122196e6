"""The shots of a seismic acquisition through one context: after fd_reset and new model, sources
and receivers (the same counts, so the device buffers and the captured step
graphs are reused; or other counts, so they are rebuilt) a shot gives bitwise
the result of a fresh context, and that result matches the FP64 oracle."""

import numpy as np
import pytest

from helpers import oracle_acoustic, rel_l2, small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _load(s, p):
    s.set_model(p["m"], p["damp"])
    s.set_sources(p["src_coords"], p["wavelet"])
    s.set_receivers(p["rec_coords"])


def _moved(p, seed):
    """The same counts with another geometry and wavelet: coordinates shifted
    by up to 4 cells (kept inside the grid), the wavelet delayed and scaled."""
    rng = np.random.default_rng(seed)
    h = np.asarray(p["spacing"], np.float64)
    top = (np.asarray(p["shape"]) - 1) * h
    q = dict(p)
    for key in ("src_coords", "rec_coords"):
        shift = rng.uniform(-4, 4, size=len(h)) * h
        q[key] = np.clip(p[key] + shift, 0, top).astype(np.float32)
    q["wavelet"] = (0.7 * np.roll(p["wavelet"], 9, axis=0)).astype(np.float32)
    return q


def _fresh(p, nt):
    from paper_1906_10811_b300 import Solver
    with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic") as s:
        _load(s, p)
        s.run(nt)
        return s.read()


@pytest.mark.parametrize("shape", [(40, 36, 45), (70, 83)])
def test_shots_in_one_context_match_fresh_contexts(shape):
    from paper_1906_10811_b300 import Solver
    nt = 150  # more than one captured chunk of steps
    a = small_problem(shape, 8, nt, nrec=12, seed=11)
    b = _moved(small_problem(shape, 8, nt, nrec=12, seed=12), 5)   # same counts as a
    c = small_problem(shape, 8, nt, nrec=7, seed=13)    # another receiver count
    assert not np.array_equal(a["src_coords"], b["src_coords"])
    assert not np.array_equal(a["rec_coords"], b["rec_coords"])
    assert not np.array_equal(a["wavelet"], b["wavelet"])
    refs = {k: _fresh(p, nt) for k, p in (("a", a), ("b", b), ("c", c))}
    with Solver(a["shape"], a["spacing"], 8, a["dt"], "acoustic") as s:
        for key, p in (("a", a), ("b", b), ("b", b), ("c", c), ("a", a)):
            _load(s, p)
            s.reset()
            s.run(nt)
            u, rec = s.read()
            assert np.array_equal(u, refs[key][0]), key
            assert np.array_equal(rec, refs[key][1]), key
    # and the shot that reused the buffers is the oracle's shot
    o = oracle_acoustic(b, nt)
    assert rel_l2(refs["b"][0], o["u"]) < 1e-4
    assert rel_l2(refs["b"][1], o["rec"]) < 1e-4


def test_reset_restarts_from_rest():
    from paper_1906_10811_b300 import Solver
    p = small_problem((33, 30, 37), 4, 60, nrec=5, seed=3)
    u0, rec0 = _fresh(p, 60)
    with Solver(p["shape"], p["spacing"], 4, p["dt"], "acoustic") as s:
        _load(s, p)
        s.set_field(np.full(p["shape"], 0.5, np.float32))
        s.run(25)
        s.reset()
        assert s.steps == 0
        u, rec = s.read()
        assert not u.any() and rec.shape[0] == 1 and not rec.any()
        s.run(60)
        u, rec = s.read()
    assert np.array_equal(u, u0) and np.array_equal(rec, rec0)


def test_reset_diffusion_zero_field():
    from paper_1906_10811_b300 import Solver
    with Solver((20, 24, 28), (1.0, 1.0, 1.0), 4, 0.05, "diffusion") as s:
        s.set_field(np.ones((20, 24, 28), np.float32))
        s.run(3)
        s.reset()
        s.run(2)
        u, _ = s.read()
    assert not u.any()


@pytest.mark.parametrize("shape", [(34, 31, 40), (90, 77)])
def test_model_upload_overlapping_a_run(shape):
    """fd_set_model while a shot's steps are in flight: they finish with the old
    coefficients, and the next shot runs on the new model."""
    from paper_1906_10811_b300 import Solver
    nt = 90
    a = small_problem(shape, 8, nt, nrec=6, seed=21)
    b = small_problem(shape, 8, nt, nrec=6, seed=22)
    assert not np.array_equal(a["m"], b["m"])
    ref_a, ref_b = _fresh(a, nt), _fresh(b, nt)
    with Solver(a["shape"], a["spacing"], 8, a["dt"], "acoustic") as s:
        _load(s, a)
        s.reset()
        s.run(nt)                      # queued; not waited for
        s.set_model(b["m"], b["damp"])
        u, rec = s.read()
        assert np.array_equal(u, ref_a[0]) and np.array_equal(rec, ref_a[1])
        s.set_sources(b["src_coords"], b["wavelet"])
        s.set_receivers(b["rec_coords"])
        s.reset()
        s.run(nt)
        u, rec = s.read()
        assert np.array_equal(u, ref_b[0]) and np.array_equal(rec, ref_b[1])
