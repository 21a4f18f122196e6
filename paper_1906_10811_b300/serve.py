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
    """Shots as library contexts in one ``fd_batch`` (the real device)."""

    def __init__(self, space_order):
        from .solver import Batch
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


class Server:
    """Continuous-batching server.

    ``hbm_budget``: device bytes the admitted shots may hold together;
    ``max_members``: batch slots; ``ticks_per_round``: most steps per batch run
    between admission points (a round also ends when a member finishes).
    """

    def __init__(self, backend, hbm_budget, max_members=64, ticks_per_round=32,
                 clock=time.perf_counter, sleep=time.sleep):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_members = int(max_members)
        self.ticks = int(ticks_per_round)
        self.clock = clock
        self.sleep = sleep
        self.log = []          # (event, request id, time) for tests and traces

    def serve(self, requests):
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.id)))
        for r in pending:
            if self.backend.footprint(r) > self.budget:
                raise ValueError(f"shot {r.id} needs more device memory than the budget")
        active = {}            # id -> [request, handle, steps done, footprint, admitted time]
        left = []              # shots that left the batch in the last round, to collect
        used = 0               # footprint held on the device (freed when collected)
        results = []
        t0 = self.clock()
        while pending or active or left:
            now = self.clock() - t0
            # admit arrivals, first come first served, while memory and slots allow
            while (pending and pending[0].arrival <= now and len(active) < self.max_members):
                r = pending[0]
                fp = self.backend.footprint(r)
                if used + fp > self.budget:
                    break
                pending.popleft()
                h = self.backend.start(r)
                self.backend.add(h)
                used += fp
                active[r.id] = [r, h, 0, fp, self.clock() - t0]
                self.log.append(("admit", r.id, self.clock() - t0))
            if not active and not left:
                wait = pending[0].arrival - (self.clock() - t0)
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
                    finished.append((r, h, fp, adm))
            for r, h, fp, adm in left:
                rec = self.backend.collect(h)
                used -= fp
                t = self.clock() - t0
                results.append(ShotResult(r.id, rec, r.arrival, adm, t))
                self.log.append(("finish", r.id, t))
            left = finished
        return sorted(results, key=lambda x: x.id)


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
