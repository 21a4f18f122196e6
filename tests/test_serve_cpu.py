"""Scheduling policy of the continuous-batching server, with a simulated
backend and clock (no GPU): first-come-first-served admission under the HBM
budget and slot limit, admission while other shots run, exact step counts,
retirement and latency accounting."""

from paper_1906_10811_b300.serve import Server, ShotRequest, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeBackend:
    """Shots cost `size` units of memory; a tick costs 1e-3 s per member."""

    def __init__(self, clock):
        self.clock = clock
        self.members = {}
        self.left = {}
        self.used = 0
        self.peak_used = 0
        self.peak_members = 0

    def footprint(self, req):
        return req.problem["size"]

    def start(self, req):
        return req

    def add(self, h):
        self.members[h.id] = [h, 0]
        self.used += h.problem["size"]
        self.peak_used = max(self.peak_used, self.used)
        self.peak_members = max(self.peak_members, len(self.members))

    def run(self, n):
        for m in self.members.values():
            m[1] += n
            assert m[1] <= m[0].problem["nt"], "a shot ran past its end"
        self.clock.t += 1e-3 * n * len(self.members)

    def leave(self, h):
        steps = self.members.pop(h.id)[1]
        assert steps == h.problem["nt"]
        self.left[h.id] = steps

    def collect(self, h):
        steps = self.left.pop(h.id)
        self.used -= h.problem["size"]
        return steps


def _reqs(spec):
    return [ShotRequest(i, a, {"size": s, "nt": nt}) for i, (a, s, nt) in enumerate(spec)]


def test_budget_slots_and_fifo():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs([(0.0, 4, 50), (0.0, 4, 30), (0.0, 4, 20), (0.001, 2, 10), (0.5, 1, 5)])
    srv = Server(be, hbm_budget=10, max_members=3, ticks_per_round=8, clock=clk, sleep=clk.sleep)
    res = srv.serve(reqs)
    assert [r.id for r in res] == [0, 1, 2, 3, 4]
    assert all(r.traces == reqs[r.id].problem["nt"] for r in res)
    assert be.peak_used <= 10 and be.peak_members <= 3
    admits = [rid for ev, rid, _ in srv.log if ev == "admit"]
    assert admits == sorted(admits)                       # first come, first served
    for r in res:
        assert r.arrival <= r.admitted <= r.finished


def test_continuous_admission_while_running():
    """A shot that arrives while a long one runs joins before the long one ends."""
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = _reqs([(0.0, 1, 1000), (0.05, 1, 10)])
    srv = Server(be, hbm_budget=100, ticks_per_round=16, clock=clk, sleep=clk.sleep)
    res = srv.serve(reqs)
    t_admit_1 = [t for ev, rid, t in srv.log if ev == "admit" and rid == 1][0]
    t_finish_0 = [t for ev, rid, t in srv.log if ev == "finish" and rid == 0][0]
    t_finish_1 = [t for ev, rid, t in srv.log if ev == "finish" and rid == 1][0]
    assert t_admit_1 < t_finish_0 and t_finish_1 < t_finish_0
    assert res[1].latency < 0.1


def test_oversized_request_rejected_and_idle_wait():
    clk = FakeClock()
    be = FakeBackend(clk)
    srv = Server(be, hbm_budget=5, clock=clk, sleep=clk.sleep)
    try:
        srv.serve(_reqs([(0.0, 6, 10)]))
        raise AssertionError("oversized request accepted")
    except ValueError:
        pass
    res = srv.serve(_reqs([(2.0, 1, 4)]))                 # server idles until the arrival
    assert res[0].admitted >= 2.0
    s = summarize(res)
    assert s["shots"] == 1 and s["p99_s"] >= s["p50_s"] > 0


def _reqs_pts(spec):
    """(arrival, size, nt, points) per request."""
    return [ShotRequest(i, a, {"size": s, "nt": nt, "points": pts})
            for i, (a, s, nt, pts) in enumerate(spec)]


def test_shortest_work_first_admission():
    clk = FakeClock()
    be = FakeBackend(clk)
    # all arrived at once, one slot: admitted by least points x steps
    reqs = _reqs_pts([(0.0, 1, 100, 50), (0.0, 1, 10, 10), (0.0, 1, 40, 20), (0.0, 1, 5, 1000)])
    srv = Server(be, hbm_budget=100, max_members=1, ticks_per_round=8, clock=clk,
                 sleep=clk.sleep, policy="shortest", max_wait_s=100.0)
    res = srv.serve(reqs)
    admits = [rid for ev, rid, _ in srv.log if ev == "admit"]
    assert admits == [1, 2, 0, 3]                 # work 100, 800, 5000, 5000 (tie: arrival, id)
    assert all(r.traces == reqs[r.id].problem["nt"] for r in res)


def test_ageing_bounds_the_wait_of_large_shots():
    """A large shot among a steady stream of small ones: shortest-first alone would
    keep passing it over; past max_wait it goes first and holds admission."""
    clk = FakeClock()
    be = FakeBackend(clk)
    spec = [(0.0, 1, 200, 100)] + [(0.001 * i, 1, 20, 1) for i in range(1, 200)]
    reqs = _reqs_pts(spec)
    srv = Server(be, hbm_budget=1000, max_members=2, ticks_per_round=4, clock=clk,
                 sleep=clk.sleep, policy="shortest", max_wait_s=0.05)
    res = srv.serve(reqs)
    t_admit_big = [t for ev, rid, t in srv.log if ev == "admit" and rid == 0][0]
    # admitted within max_wait plus the round in which it aged (a round here is at most
    # 4 ticks of 2 members = 8 ms)
    assert t_admit_big <= 0.05 + 0.01
    assert len(res) == 200


def test_work_cap_bounds_the_points_of_a_tick():
    clk = FakeClock()

    class PointBackend(FakeBackend):
        def __init__(self, clock):
            super().__init__(clock)
            self.points = 0
            self.peak_points = 0

        def add(self, h):
            super().add(h)
            self.points += h.problem["points"]
            self.peak_points = max(self.peak_points, self.points)
            if len(self.members) > 1:
                assert self.points <= 100, "a tick over the work cap"

        def leave(self, h):
            super().leave(h)
            self.points -= h.problem["points"]

    be = PointBackend(clk)
    reqs = _reqs_pts([(0.0, 1, 30, 60), (0.0, 1, 30, 50), (0.0, 1, 30, 30), (0.0, 1, 30, 200)])
    srv = Server(be, hbm_budget=1000, max_members=8, ticks_per_round=8, clock=clk,
                 sleep=clk.sleep, work_cap=100)
    res = srv.serve(reqs)
    assert len(res) == 4
    # the 200-point shot exceeds the cap alone: it runs only in an empty batch
    assert be.peak_points == 200
    admits = [rid for ev, rid, _ in srv.log if ev == "admit"]
    assert admits == [0, 1, 2, 3]                     # fcfs order kept under the cap


def test_setup_on_a_worker_keeps_budget_slots_and_results():
    """Shots set up on a worker thread while the batch runs: memory of shots being
    set up counts against the budget, every shot runs exactly its steps."""
    import threading
    clk = FakeClock()
    lock = threading.Lock()

    class SlowStart(FakeBackend):
        def start(self, req):
            with lock:
                return req

    be = SlowStart(clk)
    reqs = _reqs_pts([(0.0, 4, 50, 10), (0.0, 4, 30, 10), (0.0, 4, 20, 10), (0.001, 2, 10, 10),
                      (0.5, 1, 5, 10)])
    srv = Server(be, hbm_budget=10, max_members=3, ticks_per_round=8, clock=clk, sleep=clk.sleep,
                 setup_workers=1)
    res = srv.serve(reqs)
    assert [r.id for r in res] == [0, 1, 2, 3, 4]
    assert all(r.traces == reqs[r.id].problem["nt"] for r in res)
    assert be.peak_used <= 10 and be.peak_members <= 3
    for r in res:
        assert r.arrival <= r.admitted <= r.finished


def test_dispatch_joins_the_least_loaded_device():
    from paper_1906_10811_b300.serve import dispatch
    # work = points x steps; rate 1: device d is free at the sum of its shots' work
    reqs = _reqs_pts([(0.0, 1, 10, 10), (0.0, 1, 10, 1), (0.0, 1, 10, 1), (0.5, 1, 10, 1),
                      (200.0, 1, 10, 1)])
    where = dispatch(reqs, 2)
    assert where[0] == 0 and where[1] == 1   # both free at t = 0: the lower index, then the other
    assert where[2] == 1                     # device 1 frees at 10, device 0 at 100
    assert where[3] == 1                     # device 1 frees at 20 < 100
    assert where[4] == 0                     # both free by t = 200: the lower index
    assert dispatch(reqs, 1) == [0] * 5


def test_serve_multi_runs_every_shot_once_on_its_device():
    from paper_1906_10811_b300.serve import dispatch, serve_multi
    reqs = _reqs_pts([(0.0, 1, 20 + i, 1 + i % 3) for i in range(9)])
    backends = {}

    def make(d):
        clk = FakeClock()
        be = FakeBackend(clk)
        backends[d] = be
        return Server(be, hbm_budget=100, max_members=4, ticks_per_round=8, clock=clk,
                      sleep=clk.sleep)

    res = serve_multi(reqs, make, 3)
    assert [r.id for r in res] == list(range(9))
    assert all(r.traces == reqs[r.id].problem["nt"] for r in res)
    where = dispatch(reqs, 3)
    assert set(backends) == {d for d in where}
