"""z-slab domain decomposition of one acoustic grid (marshalling and scheduling only).

The paper's OPS backend targets structured blocks whose distributed-memory
partitioning (and halo exchange between partitions) is left to the OPS library
(thesis §2.2).  Here one 3-D grid is cut along z (axis 0, the slowest, so a
slab's planes are contiguous) into slabs; each slab is an ordinary library
context told its global placement (``fd_set_subdomain``), and after every step
each slab's halo of R = so/2 planes is refreshed from its neighbours' boundary
planes.  Sources and receivers are given in global coordinates: a source corner
is injected by the slab holding its node, and a receiver's trace is the sum of
the slabs' partial sums over the corners each holds.  Every step of the path
runs in the CUDA library; this module cuts the grid, orders the exchanges and
adds the partial traces (with the library's ``fd_accumulate_traces``).

Two drivers:

* :class:`SlabDecomposition` -- all slabs in this process (on one device, or on
  several with peer copies), stepped by the library's ``fd_run_slabs``;
* :class:`DistributedSlab` -- one slab per process (one process per GPU), the
  halo faces sent and received with ``torch.distributed`` (NCCL between GPUs)
  into each receiver's own halo, partial traces summed with ``all_reduce``.
"""

import bisect
import math

import numpy as np

from . import binding as B


def slab_bounds(nz, nslabs, R):
    """[(z0, z1)]: ``nslabs`` contiguous slabs of nearly equal thickness covering
    0..nz, each at least R planes thick (a halo face is R planes of one slab)."""
    if nslabs < 1:
        raise ValueError("nslabs must be >= 1")
    if nz < nslabs * max(int(R), 1):
        raise ValueError(f"{nz} planes cannot give {nslabs} slabs of at least {R} planes")
    return [(nz * s // nslabs, nz * (s + 1) // nslabs) for s in range(nslabs)]


def halo_schedule(nslabs):
    """The messages of one halo exchange: (src, face, dst, halo).

    face 0 / 1: the first / last R planes of slab src; halo 0 / 1: the halo
    below / above slab dst.  Every interior interface carries two messages."""
    out = []
    for s in range(nslabs - 1):
        out.append((s, 1, s + 1, 0))   # top planes of s -> halo below s+1
        out.append((s + 1, 0, s, 1))   # bottom planes of s+1 -> halo above s
    return out


def slab_of_plane(bounds, z):
    """Index of the slab holding global plane z."""
    starts = [b[0] for b in bounds]
    s = bisect.bisect_right(starts, z) - 1
    if s < 0 or z >= bounds[s][1]:
        raise ValueError(f"plane {z} outside the slabs")
    return s


def corner_planes(coord_z, h, nz):
    """The two z planes of a point's multilinear corners (the library's rule:
    i = floor(z/h), a point on the last plane uses i = nz-2), and their weights."""
    x = float(coord_z) / h
    last = float(nz - 1)
    tol = 1e-9 * last
    if not (-tol <= x <= last + tol):
        raise ValueError("coordinate outside the grid")
    x = min(max(x, 0.0), last)
    i = int(math.floor(x))
    f = x - i
    if i == nz - 1:
        i, f = nz - 2, 1.0
    return (i, i + 1), (1.0 - f, f)


def owners(coord_z, h, nz, bounds):
    """Slabs that hold a corner (of non-zero weight or not) of a point at z = coord_z."""
    planes, _ = corner_planes(coord_z, h, nz)
    return sorted({slab_of_plane(bounds, z) for z in planes})


def _slab_arg(a, z0, z1):
    return None if a is None else a[z0:z1]


class SlabDecomposition:
    """One acoustic grid cut into z-slabs, all driven from this process.

    ``SlabDecomposition(shape, spacing, space_order, dt, nslabs)``; arrays are
    torch CUDA tensors (device mode).  ``streams``: "shared" runs every slab on
    one stream (the caller's current one, or a private one when that is the
    legacy default stream); "separate" gives each slab its own stream, the
    exchanges then ordered by events.  ``devices``: one CUDA device index per
    slab (default: the current device for all), exchanges by peer copies.
    """

    def __init__(self, shape, spacing, space_order, dt, nslabs, streams="shared", devices=None,
                 **solver_kw):
        import torch
        from .solver import Solver
        self._torch = torch
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) != 3:
            raise ValueError("z-slabs cut a 3-D grid")
        self.R = int(space_order) // 2
        self.bounds = slab_bounds(self.shape[0], int(nslabs), self.R)
        cur = torch.cuda.current_device()
        self.devices = list(devices) if devices is not None else [cur] * len(self.bounds)
        if len(self.devices) != len(self.bounds):
            raise ValueError("one device per slab")
        shared = None
        if streams == "shared" and len(set(self.devices)) == 1:
            shared = torch.cuda.current_stream()
            if shared.cuda_stream == 0:
                shared = torch.cuda.Stream()
        self.slabs = []
        for (z0, z1), dev in zip(self.bounds, self.devices):
            with torch.cuda.device(dev):
                st = shared if shared is not None else torch.cuda.Stream(device=dev)
                s = Solver((z1 - z0,) + self.shape[1:], spacing, space_order, dt, "acoustic",
                           device=True, stream=st, **solver_kw)
                B.fd_set_subdomain(s.ctx, z0, self.shape[0])
            self.slabs.append(s)
        self.nrec = 0

    def _each(self, fn):
        torch = self._torch
        for s, dev in zip(self.slabs, self.devices):
            with torch.cuda.device(dev), torch.cuda.stream(s.stream):
                fn(s)

    def _slice_to(self, a, z0, z1, dev):
        if a is None:
            return None
        t = self._torch.as_tensor(a[z0:z1], dtype=self._torch.float32)
        return t.to(f"cuda:{dev}").contiguous()

    def _wait_caller(self):
        caller = self._torch.cuda.current_stream()
        for s in self.slabs:
            s.stream.wait_stream(caller)

    def set_model(self, m, damp=None):
        self._wait_caller()
        for s, (z0, z1), dev in zip(self.slabs, self.bounds, self.devices):
            with self._torch.cuda.device(dev), self._torch.cuda.stream(s.stream):
                s.set_model(self._slice_to(m, z0, z1, dev), self._slice_to(damp, z0, z1, dev))

    def set_field(self, u, u_prev=None):
        self._wait_caller()
        for s, (z0, z1), dev in zip(self.slabs, self.bounds, self.devices):
            with self._torch.cuda.device(dev), self._torch.cuda.stream(s.stream):
                s.set_field(self._slice_to(u, z0, z1, dev), self._slice_to(u_prev, z0, z1, dev))

    def set_sources(self, coords, wavelets):
        """Global coordinates: every slab takes the list and keeps the corners it holds."""
        self._wait_caller()
        torch = self._torch
        for s, dev in zip(self.slabs, self.devices):
            with torch.cuda.device(dev), torch.cuda.stream(s.stream):
                s.set_sources(torch.as_tensor(coords, dtype=torch.float32).to(f"cuda:{dev}"),
                              torch.as_tensor(wavelets, dtype=torch.float32).to(f"cuda:{dev}"))

    def set_receivers(self, coords):
        self._wait_caller()
        torch = self._torch
        self.nrec = 0 if coords is None else len(coords)
        for s, dev in zip(self.slabs, self.devices):
            with torch.cuda.device(dev), torch.cuda.stream(s.stream):
                s.set_receivers(torch.as_tensor(coords, dtype=torch.float32).to(f"cuda:{dev}"))

    def set_tile_config(self, **cfg):
        self._each(lambda s: s.set_tile_config(**cfg))

    def reset(self):
        self._each(lambda s: s.reset())

    def run(self, nt):
        self._wait_caller()
        B.fd_run_slabs([s.ctx for s in self.slabs], nt)
        caller = self._torch.cuda.current_stream()
        for s in self.slabs:
            caller.wait_stream(s.stream)
        return self

    @property
    def steps(self):
        return self.slabs[0].steps

    def read(self):
        """(u^n of the whole grid, traces [n+1][nrec] summed over the slabs), on the
        first slab's device."""
        torch = self._torch
        dev0 = self.devices[0]
        parts = []
        for s, dev in zip(self.slabs, self.devices):
            with torch.cuda.device(dev), torch.cuda.stream(s.stream):
                u, _ = s.read(traces=False)
            parts.append(u.to(f"cuda:{dev0}"))
        u = torch.cat(parts, dim=0)
        rec = None
        if self.nrec:
            # slab by slab, each accumulation ordered after the previous one
            caller = torch.cuda.current_stream()
            rec = torch.zeros((self.steps + 1, self.nrec), dtype=torch.float32,
                              device=f"cuda:{dev0}")
            prev = caller
            for s, dev in zip(self.slabs, self.devices):
                if dev == dev0:
                    s.stream.wait_stream(prev)
                    B.fd_accumulate_traces(s.ctx, rec)       # on the slab's stream
                    prev = s.stream
                else:
                    with torch.cuda.device(dev), torch.cuda.stream(s.stream):
                        part = torch.zeros(rec.shape, dtype=torch.float32, device=f"cuda:{dev}")
                        B.fd_accumulate_traces(s.ctx, part)
                    prev.wait_stream(s.stream)
                    with torch.cuda.stream(prev):
                        rec.add_(part.to(f"cuda:{dev0}"))
            caller.wait_stream(prev)
        return u, rec

    def close(self):
        for s in getattr(self, "slabs", []):
            s.close()
        self.slabs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class SolverSlab:
    """This process's slab as a library context (device mode): the backend of
    :class:`DistributedSlab`.  Faces are exported on the context's stream, which
    ``sync`` waits for; imports run on it after the caller's stream (where the
    received buffers become valid)."""

    def __init__(self, solver):
        import torch
        self._torch = torch
        self.solver = solver
        self.elems = B.fd_halo_elems(solver.ctx)

    def new_buffer(self):
        return self._torch.empty(self.elems, dtype=self._torch.float32, device="cuda")

    def step(self):
        self.solver.run(1)

    def export_face(self, face, buf):
        self.solver.stream.wait_stream(self._torch.cuda.current_stream())
        B.fd_halo_export(self.solver.ctx, face, buf)

    def import_halo(self, halo, buf):
        self.solver.stream.wait_stream(self._torch.cuda.current_stream())
        B.fd_halo_import(self.solver.ctx, halo, buf)

    def partial_traces(self):
        _, rec = self.solver.read(field=False)
        return rec

    def sync(self):
        self.solver.stream.synchronize()


class DistributedSlab:
    """One slab per rank of a ``torch.distributed`` group (one process per GPU).

    ``backend`` runs this rank's slab and moves its halo faces through buffers
    (:class:`SolverSlab` for the library; anything with the same methods).
    Each exchange follows :func:`halo_schedule`: a rank sends the faces its
    neighbours need and receives into its own halo buffers, then imports them.
    """

    def __init__(self, backend, rank, world, group=None):
        self.b = backend
        self.rank, self.world, self.group = rank, world, group
        self.send = {f: backend.new_buffer() for f in (0, 1)}
        self.recv = {h: backend.new_buffer() for h in (0, 1)}

    def exchange(self):
        import torch.distributed as dist
        ops, incoming = [], []
        for src, face, dst, halo in halo_schedule(self.world):
            if src == self.rank:
                self.b.export_face(face, self.send[face])
            if dst == self.rank:
                incoming.append(halo)
        self.b.sync()                     # faces exported before they are sent
        for src, face, dst, halo in halo_schedule(self.world):
            if src == self.rank:
                ops.append(dist.P2POp(dist.isend, self.send[face], dst, self.group))
            if dst == self.rank:
                ops.append(dist.P2POp(dist.irecv, self.recv[halo], src, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for halo in incoming:
            self.b.import_halo(halo, self.recv[halo])

    def run(self, nt):
        self.exchange()
        for _ in range(nt):
            self.b.step()
            self.exchange()

    def traces(self):
        """The whole grid's traces: the ranks' partial traces summed (every rank)."""
        import torch.distributed as dist
        rec = self.b.partial_traces()
        out = rec.clone()
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=self.group)
        return out
