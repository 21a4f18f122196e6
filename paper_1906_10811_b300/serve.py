"""Serving loop for shot simulations: continuous batching over the batch C ABI.

Requests (one acoustic shot each: grid, model, source, receivers, nt) arrive
over time.  The server keeps the admitted shots' wavefields resident on the
device and steps them together (``fd_batch_run``); between rounds it admits
requests that have arrived, first come first served, while their device
footprint (``fd_footprint_bytes``) fits the HBM budget and a member slot is
free, and retires shots that have finished (their traces are read back and
their memory freed, while the next round already runs).  New shots are set up
on their own CUDA streams while the batch is running, so admission overlaps
the device work.

Scheduling is separate from execution: :class:`Server` drives any backend with
the small interface of :class:`DeviceBackend`, which lets the policy be tested
without a GPU.  Every numerical step runs in the CUDA library.
"""

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class ShotRequest:
    """One shot: problem arrays as produced by ``fdsynth.acoustic_problem``."""
    id: int
    arrival: float          # seconds after the stream starts
    problem: dict           # shape, spacing, so, dt, nt, m, damp, src_coords, wavelet, rec_coords


@dataclasses.dataclass
class ShotResult:
    id: int
    traces: np.ndarray
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self):
        return self.finished - self.arrival


class DeviceBackend:
    """Shots as library contexts in one ``fd_batch`` (the real device).

    ``device``: the CUDA device the shots run on, made current on the calling
    thread (the library creates contexts on the current device)."""

    def __init__(self, space_order, device=None):
        from .solver import Batch
        if device is not None:
            import torch
            torch.cuda.set_device(device)
        self.batch = Batch(space_order)

    def footprint(self, req):
        from .binding import fd_footprint_bytes
        p = req.problem
        return fd_footprint_bytes(p["shape"], p["so"], len(p["rec_coords"]), p["nt"],
                                  len(p["src_coords"]))

    def start(self, req):
        """Create the shot's context (own stream) and upload its inputs."""
        from .solver import Solver
        p = req.problem
        s = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic")
        s.set_model(p["m"], p["damp"])
        s.set_sources(p["src_coords"], p["wavelet"])
        s.set_receivers(p["rec_coords"])
        return s

    def add(self, handle):
        self.batch.add(handle)

    def run(self, nticks):
        self.batch.run(nticks)

    def leave(self, handle):
        """Take a finished shot out of the batch (no wait: later runs skip it)."""
        self.batch.remove(handle)

    def collect(self, handle):
        """Read the traces of a shot that left (waits for its last step) and free it."""
        _, rec = handle.read(field=False)
        handle.close()
        return rec

    def close(self):
        self.batch.close()


def shot_work(req):
    """Grid-point updates of a shot (points × steps): the service-time estimate."""
    return shot_points(req) * int(req.problem["nt"])


def shot_points(req):
    """Grid points one tick of the shot updates (its share of a batch tick)."""
    p = req.problem
    return int(np.prod(p["shape"])) if "shape" in p else int(p.get("points", 1))


class Server:
    """Continuous-batching server.

    ``hbm_budget``: device bytes the admitted shots may hold together;
    ``max_members``: batch slots; ``ticks_per_round``: most steps per batch run
    between admission points (a round also ends when a member finishes).

    Admission order (``policy``): "fcfs" admits arrived requests in arrival
    order and stops at the first that does not fit; "shortest" admits the
    arrived request with the least work (points × steps) first, except that a
    request waiting longer than ``max_wait_s`` goes ahead of all younger ones
    (oldest first) and, if it does not fit, holds admission until it does, so
    no request waits without bound.  ``work_cap`` (grid points, 0 = none)
    bounds the points one batch tick updates: every member advances once per
    tick, so the tick time, and with it every member's latency, grows with the
    work admitted beside it; a request is admitted while the batch stays under
    the cap (always when the batch is empty).
    """

    def __init__(self, backend, hbm_budget, max_members=64, ticks_per_round=32,
                 clock=time.perf_counter, sleep=time.sleep, policy="fcfs", max_wait_s=0.25,
                 work_cap=0, setup_workers=0):
        if policy not in ("fcfs", "shortest"):
            raise ValueError(f"unknown admission policy {policy!r}")
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_members = int(max_members)
        self.ticks = int(ticks_per_round)
        self.clock = clock
        self.sleep = sleep
        self.policy = policy
        self.max_wait = float(max_wait_s)
        self.work_cap = int(work_cap)
        self.setup_workers = int(setup_workers)
        self.log = []          # (event, request id, time) for tests and traces

    def _candidates(self, pending, now):
        """Arrived requests in the order admission considers them, and how many at
        the head of that order no later request may pass (all of them under fcfs;
        the aged ones under shortest-first)."""
        arrived = [r for r in pending if r.arrival <= now]
        if self.policy == "fcfs":
            return arrived, len(arrived)
        aged = sorted((r for r in arrived if now - r.arrival > self.max_wait),
                      key=lambda r: (r.arrival, r.id))
        young = sorted((r for r in arrived if now - r.arrival <= self.max_wait),
                       key=lambda r: (shot_work(r), r.arrival, r.id))
        return aged + young, len(aged)

    def serve(self, requests):
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.id)))
        for r in pending:
            if self.backend.footprint(r) > self.budget:
                raise ValueError(f"shot {r.id} needs more device memory than the budget")
        active = {}            # id -> [request, handle, steps done, footprint, admitted time]
        starting = {}          # id -> [request, future of its set-up, footprint]
        left = []              # shots that left the batch in the last round, to collect
        used = 0               # footprint held on the device (freed when collected)
        points = 0             # grid points one tick of the admitted shots updates
        results = []
        pool = None
        if self.setup_workers > 0:
            import concurrent.futures
            pool = concurrent.futures.ThreadPoolExecutor(max_workers=self.setup_workers)
        t0 = self.clock()

        def join(r, h):
            self.backend.add(h)
            active[r.id] = [r, h, 0, self.backend.footprint(r), self.clock() - t0]
            self.log.append(("admit", r.id, self.clock() - t0))

        try:
            while pending or active or left or starting:
                # shots whose set-up finished join the batch
                for rid in [rid for rid, st in starting.items() if st[1].done()]:
                    r, fut, _ = starting.pop(rid)
                    join(r, fut.result())
                now = self.clock() - t0
                # admit arrivals in policy order while memory, slots and the work cap allow
                cands, nblock = self._candidates(pending, now)
                for i, r in enumerate(cands):
                    if len(active) + len(starting) >= self.max_members:
                        break
                    fp = self.backend.footprint(r)
                    pts = shot_points(r)
                    busy = active or starting
                    fits = used + fp <= self.budget and (
                        not self.work_cap or not busy or points + pts <= self.work_cap)
                    if not fits:
                        if i < nblock:
                            break          # a request nobody may pass waits for room
                        continue
                    pending.remove(r)
                    used += fp
                    points += pts
                    if pool is None:
                        join(r, self.backend.start(r))
                    else:              # set up on a worker while the batch runs
                        starting[r.id] = [r, pool.submit(self.backend.start, r), fp]
                if not active and not left:
                    if starting:       # nothing to run until a set-up finishes
                        next(iter(starting.values()))[1].result()
                        continue
                    if pending:
                        wait = min(r.arrival for r in pending) - (self.clock() - t0)
                        if wait > 0:
                            self.sleep(min(wait, 0.05))
                    continue
                # queue the next round first, then collect the shots that finished in
                # the previous one: reading their traces overlaps this round's work
                finished = []
                if active:
                    n = min([self.ticks] + [a[0].problem["nt"] - a[2] for a in active.values()])
                    self.backend.run(n)
                    for a in active.values():
                        a[2] += n
                    for rid in [rid for rid, a in active.items() if a[2] == a[0].problem["nt"]]:
                        r, h, _, fp, adm = active.pop(rid)
                        self.backend.leave(h)
                        points -= shot_points(r)
                        finished.append((r, h, fp, adm))
                for r, h, fp, adm in left:
                    rec = self.backend.collect(h)
                    used -= fp
                    t = self.clock() - t0
                    results.append(ShotResult(r.id, rec, r.arrival, adm, t))
                    self.log.append(("finish", r.id, t))
                left = finished
        finally:
            if pool is not None:
                pool.shutdown(wait=True)
        return sorted(results, key=lambda x: x.id)


def dispatch(requests, ndev, rate=None):
    """Place each request on one of ``ndev`` devices: the one predicted to be free
    first when it arrives (join the least-loaded queue).  A device's predicted free
    time moves to max(free, arrival) + work / rate, with work = points × steps
    (:func:`shot_work`) and ``rate`` its update rate (1 when not given: only the
    order matters).  Returns one device index per request, in request order."""
    rate = float(rate or 1.0)
    free = [0.0] * ndev
    out = {}
    for r in sorted(requests, key=lambda r: (r.arrival, r.id)):
        d = min(range(ndev), key=lambda k: (max(free[k], r.arrival), k))
        free[d] = max(free[d], r.arrival) + shot_work(r) / rate
        out[r.id] = d
    return [out[r.id] for r in requests]


def serve_multi(requests, make_server, ndev, rate=None):
    """Serve a stream on ``ndev`` devices, shots being replicas: :func:`dispatch`
    splits the requests, ``make_server(d)`` builds device d's :class:`Server`
    (called on d's worker thread, so a backend can make d current there), and the
    servers run concurrently, one host thread per device.  Returns every result,
    sorted by request id."""
    import threading
    where = dispatch(requests, ndev, rate)
    parts = [[r for r, d in zip(requests, where) if d == k] for k in range(ndev)]
    results, errors = [None] * ndev, []

    def work(k):
        try:
            srv = make_server(k)
            results[k] = srv.serve(parts[k]) if parts[k] else []
        except BaseException as e:          # re-raised on the calling thread
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(ndev)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    return sorted((x for part in results for x in part), key=lambda x: x.id)


def serve_sequential(requests, clock=time.perf_counter, sleep=time.sleep):
    """Baseline: one shot at a time in arrival order, each run alone with fd_run."""
    from .solver import Solver
    out = []
    t0 = clock()
    for r in sorted(requests, key=lambda r: (r.arrival, r.id)):
        while clock() - t0 < r.arrival:
            sleep(min(r.arrival - (clock() - t0), 0.05))
        start = clock() - t0
        p = r.problem
        with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic") as s:
            s.set_model(p["m"], p["damp"])
            s.set_sources(p["src_coords"], p["wavelet"])
            s.set_receivers(p["rec_coords"])
            s.run(p["nt"])
            _, rec = s.read(field=False)
        out.append(ShotResult(r.id, rec, r.arrival, start, clock() - t0))
    return sorted(out, key=lambda x: x.id)


def summarize(results):
    """shots/s over the whole stream and latency percentiles (seconds)."""
    lat = np.array([r.latency for r in results])
    span = max(r.finished for r in results) - min(r.arrival for r in results)
    return {"shots": len(results), "seconds": span, "shots_per_s": len(results) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean())}
