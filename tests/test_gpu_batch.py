"""Batched shots through the C ABI: a mix of 2-D and 3-D shots of different
sizes, admitted and retired between runs, gives every shot bitwise the result
of running it alone (same kernels' arithmetic, fixed reduction orders), and the
results match the FP64 oracle."""

import numpy as np
import pytest

import fdsynth
from helpers import oracle_acoustic, rel_l2, small_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _solver(p, stream=None):
    from paper_1906_10811_b300 import Solver
    s = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic")
    s.set_model(p["m"], p["damp"])
    s.set_sources(p["src_coords"], p["wavelet"])
    s.set_receivers(p["rec_coords"])
    return s


def _alone(p, nt):
    s = _solver(p)
    s.run(nt)
    u, rec = s.read()
    up = s.read_prev()
    s.close()
    return u, up, rec


SHOTS = [((30, 26, 41), 90, 1), ((61, 53), 120, 2), ((44, 37, 35), 70, 3), ((17, 130), 100, 4),
         ((25, 29, 33), 110, 5)]


def test_batch_matches_alone_runs_with_joins_and_leaves():
    from paper_1906_10811_b300 import Batch
    probs = [small_problem(shape, 8, nt, nrec=9, seed=seed) for shape, nt, seed in SHOTS]
    refs = [_alone(p, p["nt"]) for p in probs]
    batch = Batch(8)
    solvers = [None] * len(probs)
    done = [0] * len(probs)
    results = [None] * len(probs)
    # admission schedule: shot i joins at tick 15*i; runs go in chunks of 13 ticks
    tick = 0
    while any(r is None for r in results):
        for i, p in enumerate(probs):
            if solvers[i] is None and results[i] is None and tick >= 15 * i:
                solvers[i] = _solver(p)
                batch.add(solvers[i])
        active = [i for i in range(len(probs)) if solvers[i] is not None]
        n = min([13] + [probs[i]["nt"] - done[i] for i in active])
        batch.run(n)
        tick += n
        for i in active:
            done[i] += n
            if done[i] == probs[i]["nt"]:
                s = solvers[i]
                batch.remove(s)
                u, rec = s.read()
                results[i] = (u, s.read_prev(), rec)
                s.close()
                solvers[i] = None
    assert batch.kernel_launches > 0
    batch.close()
    for (u, up, rec), (ru, rup, rrec) in zip(results, refs):
        assert np.array_equal(u, ru)
        assert np.array_equal(up, rup)
        assert np.array_equal(rec, rrec)


def test_batch_results_match_oracle():
    from paper_1906_10811_b300 import Batch
    probs = [small_problem(shape, 8, nt, nrec=9, seed=seed) for shape, nt, seed in SHOTS[:3]]
    nt = 60
    with Batch(8) as batch:
        ss = [_solver(p) for p in probs]
        for s in ss:
            batch.add(s)
        batch.run(nt)
        for p, s in zip(probs, ss):
            u, rec = s.read()
            o = oracle_acoustic(p, nt)
            assert rel_l2(u, o["u"]) <= 1e-4 and rel_l2(rec, o["rec"]) <= 1e-4
        for s in ss:
            batch.remove(s)
            s.close()


def test_batch_rejects_wrong_members():
    from paper_1906_10811_b300 import Batch, FdError, Solver
    p = small_problem((20, 21, 22), 4, 10)
    with Batch(8) as batch:
        s = Solver(p["shape"], p["spacing"], 4, p["dt"], "acoustic")
        s.set_model(p["m"], p["damp"])
        with pytest.raises(FdError):
            batch.add(s)                                   # space order 4 in a so-8 batch
        s.close()
        d = Solver((20, 20), (1.0, 1.0), 8, 0.01, "diffusion")
        with pytest.raises(FdError):
            batch.add(d)
        d.close()
        # 3-D members share their spacing (their weights are one kernel parameter)
        q = small_problem((20, 21, 22), 8, 10)
        a = Solver(q["shape"], q["spacing"], 8, q["dt"], "acoustic")
        a.set_model(q["m"], q["damp"])
        batch.add(a)
        h2 = tuple(1.1 * h for h in q["spacing"])
        b = Solver(q["shape"], h2, 8, q["dt"], "acoustic")
        b.set_model(q["m"], q["damp"])
        with pytest.raises(FdError) as e:
            batch.add(b)
        assert "spacing" in str(e.value)
        batch.remove(a)
        a.close()
        b.close()


def test_footprint_covers_allocations():
    """The admission measure bounds what a shot takes from the device (the
    stream-ordered pool reserves in chunks of tens of MB: one chunk of slack)."""
    import torch
    from paper_1906_10811_b300 import fd_footprint_bytes
    p = small_problem((192, 160, 176), 8, 200, nrec=32)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    s = _solver(p)
    s.run(200)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    fp = fd_footprint_bytes(p["shape"], 8, 32, 200)
    s.close()
    assert fp > 0
    assert used <= fp * 1.1 + (64 << 20)


def test_batch_runs_of_every_length_match_alone():
    """Runs of 1..64+ ticks (launched, then replayed from captured graphs) give
    bitwise the alone results."""
    from paper_1906_10811_b300 import Batch
    probs = [small_problem(shape, 8, nt, nrec=6, seed=seed)
             for shape, nt, seed in [((27, 33, 38), 160, 11), ((45, 52), 160, 12)]]
    refs = [_alone(p, p["nt"]) for p in probs]
    batch = Batch(8)
    solvers = [_solver(p) for p in probs]
    for s in solvers:
        batch.add(s)
    done = 0
    for n in (1, 2, 3, 2, 5, 8, 13, 8, 21, 33, 64):
        batch.run(n)
        done += n
    assert done == 160
    for s, ref in zip(solvers, refs):
        batch.remove(s)
        u, rec = s.read()
        up = s.read_prev()
        assert np.array_equal(u, ref[0]) and np.array_equal(up, ref[1])
        assert np.array_equal(rec, ref[2])
        s.close()
    batch.close()
