"""The serving loop on the device: a small Poisson stream of 2-D and 3-D shots
under an HBM budget that forces queueing; every served shot's traces equal
those of the shot run alone (bitwise) and those of the sequential baseline."""

import numpy as np
import pytest

import fdsynth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def test_served_shots_equal_alone_runs():
    from paper_1906_10811_b300 import fd_footprint_bytes
    from paper_1906_10811_b300.serve import (DeviceBackend, Server, ShotRequest, serve_sequential,
                                             summarize)
    stream = fdsynth.serving_stream(nshots=10, seed=7, mean_gap_s=0.002, sizes2d=(60, 140),
                                    sizes3d=(24, 56), nt_range=(40, 120), nrec_range=(8, 24))
    reqs = [ShotRequest(i, a, p) for i, a, p in stream]
    fps = [fd_footprint_bytes(p["shape"], 8, len(p["rec_coords"]), p["nt"]) for _, _, p in stream]
    budget = int(sum(sorted(fps)[-4:]))                  # about four shots at a time
    be = DeviceBackend(8)
    srv = Server(be, hbm_budget=budget, max_members=6, ticks_per_round=16)
    served = srv.serve(reqs)
    be.close()
    alone = serve_sequential(reqs)
    for a, b in zip(served, alone):
        assert a.id == b.id
        assert np.array_equal(a.traces, b.traces)
        assert np.abs(a.traces).max() > 0
    admits = [rid for ev, rid, _ in srv.log if ev == "admit"]
    assert admits == sorted(admits)
    s = summarize(served)
    assert s["shots"] == 10 and s["shots_per_s"] > 0


@pytest.mark.parametrize("policy,cap", [("fcfs", 600_000), ("shortest", 0)])
def test_policies_and_two_servers_keep_every_shot_bitwise(policy, cap):
    """Admission with a tick work cap or shortest-work-first, and the stream split over
    two servers running concurrently (both on this GPU, each on its own host thread, as
    one server per device would run): every shot's traces are those of the shot alone."""
    from paper_1906_10811_b300.serve import (DeviceBackend, Server, ShotRequest, serve_multi,
                                             serve_sequential)
    stream = fdsynth.serving_stream(nshots=8, seed=11, mean_gap_s=0.002, sizes2d=(60, 140),
                                    sizes3d=(24, 56), nt_range=(40, 100), nrec_range=(8, 24))
    reqs = [ShotRequest(i, a, p) for i, a, p in stream]
    alone = serve_sequential(reqs)
    be = DeviceBackend(8)
    srv = Server(be, hbm_budget=1 << 33, max_members=6, ticks_per_round=16, policy=policy,
                 max_wait_s=0.01, work_cap=cap)
    served = srv.serve(reqs)
    be.close()
    bes = []

    def make(d):
        b = DeviceBackend(8, device=0)
        bes.append(b)
        return Server(b, hbm_budget=1 << 33, max_members=6, ticks_per_round=16, policy=policy,
                      work_cap=cap)

    multi = serve_multi(reqs, make, 2)
    for b in bes:
        b.close()
    for a, b, c in zip(served, alone, multi):
        assert a.id == b.id == c.id
        assert np.array_equal(a.traces, b.traces) and np.array_equal(c.traces, b.traces)
