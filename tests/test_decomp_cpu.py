"""The z-slab decomposition's host logic on CPU.

* The partition, the exchange schedule and the corner-ownership rule.
* The one-process-per-GPU driver (``DistributedSlab``) over two gloo ranks:
  each rank holds one z-slab of an acoustic grid, stepped here by the FP64
  oracle on the slab plus its halo planes (a stand-in for the library context,
  with the same export/import/step interface), and the halo faces travel with
  torch.distributed.  The gathered field must be bitwise the oracle's run on
  the whole grid (every point's update reads the same values), and the traces,
  summed over the ranks from partial sums over the corners each rank holds,
  must match the whole-grid traces to rounding.
"""

import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_partition_and_schedule():
    from paper_1906_10811_b300.decomp import halo_schedule, slab_bounds, slab_of_plane
    b = slab_bounds(41, 4, 4)
    assert b == [(0, 10), (10, 20), (20, 30), (30, 41)]
    assert all(z1 - z0 >= 4 for z0, z1 in b)
    assert [slab_of_plane(b, z) for z in (0, 9, 10, 29, 30, 40)] == [0, 0, 1, 2, 3, 3]
    with pytest.raises(ValueError):
        slab_bounds(15, 4, 4)                    # a slab thinner than the halo
    s = halo_schedule(3)
    assert s == [(0, 1, 1, 0), (1, 0, 0, 1), (1, 1, 2, 0), (2, 0, 1, 1)]
    assert halo_schedule(1) == []
    # every interface sends each side's boundary face into the other's facing halo
    for src, face, dst, halo in s:
        assert abs(src - dst) == 1 and face == (1 if dst > src else 0) and halo == 1 - face


def test_corner_planes_follow_the_oracle_corners():
    from oracle import core as oracle
    from paper_1906_10811_b300.decomp import corner_planes, owners, slab_bounds
    shape, h = (23, 7, 6), 10.0
    rng = np.random.default_rng(4)
    zs = list(rng.uniform(0, (shape[0] - 1) * h, 200)) + [0.0, (shape[0] - 1) * h, 10 * h,
                                                           9.5 * h]
    bounds = slab_bounds(shape[0], 3, 2)
    for z in zs:
        node, w = oracle.corners(shape, (h,) * 3, np.array([z, 3 * h, 2.5 * h]))
        planes = sorted({int(n) // (shape[1] * shape[2]) for n in node})
        (i0, i1), (w0, w1) = corner_planes(z, h, shape[0])
        assert planes == [i0, i1]
        got = owners(z, h, shape[0], bounds)
        assert got == sorted({b for b, (a, c) in enumerate(bounds) for p in (i0, i1) if a <= p < c})
        assert abs(w0 + w1 - 1.0) < 1e-12


class OracleSlab:
    """One rank's slab stepped by the FP64 oracle on the slab and its halo planes."""

    def __init__(self, p, bounds, rank):
        from paper_1906_10811_b300.decomp import corner_planes
        self.p = p
        self.z0, self.z1 = bounds[rank]
        self.R = p["so"] // 2
        nz, ny, nx = p["shape"]
        self.nz, self.plane = nz, ny * nx
        R, z0, z1 = self.R, self.z0, self.z1
        g = np.clip(np.arange(z0 - R, z1 + R), 0, nz - 1)
        inside = (np.arange(z0 - R, z1 + R) >= 0) & (np.arange(z0 - R, z1 + R) < nz)
        self.outside = ~inside
        self.m = p["m"].astype(np.float64)[g]
        self.damp = p["damp"].astype(np.float64)[g]
        self.u = np.zeros((z1 - z0 + 2 * R, ny, nx))
        self.up = np.zeros_like(self.u)
        h = p["spacing"][0]
        mine = [j for j, c in enumerate(p["src_coords"])
                if any(z0 <= q < z1 for q in corner_planes(c[0], h, nz)[0])]
        self.src = np.array(p["src_coords"], np.float64)[mine]
        self.src[:, 0] -= (z0 - R) * h
        self.wav = np.array(p["wavelet"], np.float64)[:, mine]
        self.n = 0
        self.rec = [self._partial()]

    def _partial(self):
        from oracle import core as oracle
        out = np.zeros(len(self.p["rec_coords"]))
        for k, c in enumerate(self.p["rec_coords"]):
            node, w = oracle.corners(self.p["shape"], self.p["spacing"], c)
            for nd, wt in zip(node, w):
                z, r = divmod(int(nd), self.plane)
                if self.z0 <= z < self.z1:
                    out[k] += wt * self.u.reshape(self.u.shape[0], -1)[z - self.z0 + self.R, r]
        return out

    def new_buffer(self):
        import torch
        return torch.zeros(self.R * self.plane, dtype=torch.float64)

    def step(self):
        from oracle import core as oracle
        u, up, _ = oracle.acoustic(self.m, self.p["dt"], self.p["spacing"], self.p["so"], 1,
                                   damp=self.damp, u_cur=self.u, u_prev=self.up,
                                   src_coords=self.src if len(self.src) else None,
                                   wavelet=self.wav if len(self.src) else None, n0=self.n)
        u[self.outside] = 0.0          # beyond the grid: the zero halo
        self.u, self.up = u, up
        self.n += 1
        self.rec.append(self._partial())

    def export_face(self, face, buf):
        R = self.R
        planes = self.u[R:2 * R] if face == 0 else self.u[-2 * R:-R]
        buf.copy_(__import__("torch").from_numpy(planes.reshape(-1).copy()))

    def import_halo(self, halo, buf):
        R = self.R
        data = buf.numpy().reshape((R,) + self.u.shape[1:])
        if halo == 0:
            self.u[:R] = data
        else:
            self.u[-R:] = data

    def sync(self):
        pass

    def partial_traces(self):
        import torch
        return torch.from_numpy(np.array(self.rec))

    def interior(self):
        return self.u[self.R:-self.R]


def _problem():
    import fdsynth
    shape, so, nt = (20, 18, 22), 4, 25
    p = fdsynth.acoustic_problem(n=shape, ndim=3, so=so, nbl=4, nt=nt, nrec=10, seed=3, f0=0.05)
    h = p["spacing"][0]
    extra_src = np.array([[10 * h, 8 * h, 9 * h], [9.5 * h, 9 * h, 12 * h]], np.float32)
    p["src_coords"] = np.vstack([p["src_coords"], extra_src]).astype(np.float32)
    p["wavelet"] = np.repeat(p["wavelet"], 3, axis=1) * np.array([1.0, 0.7, -0.4], np.float32)
    extra_rec = np.array([[9.6 * h, 5 * h, 7 * h], [9.0 * h, 11 * h, 13 * h]], np.float32)
    p["rec_coords"] = np.vstack([p["rec_coords"], extra_rec]).astype(np.float32)
    return p


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1906_10811_b300.decomp import DistributedSlab, slab_bounds
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _problem()
    bounds = slab_bounds(p["shape"][0], world, p["so"] // 2)
    slab = OracleSlab(p, bounds, rank)
    drv = DistributedSlab(slab, rank, world)
    drv.run(10)
    drv.run(p["nt"] - 10)
    rec = drv.traces().numpy()
    fields = [None] * world
    dist.all_gather_object(fields, slab.interior())
    if rank == 0:
        out.put((np.concatenate(fields, axis=0), rec))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_whole_grid():
    from oracle import core as oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    u, rec = q.get(timeout=300)
    for pr in procs:
        pr.join(120)
        assert pr.exitcode == 0
    p = _problem()
    ou, _, orec = oracle.acoustic(p["m"], p["dt"], p["spacing"], p["so"], p["nt"], damp=p["damp"],
                                  src_coords=p["src_coords"], wavelet=p["wavelet"],
                                  rec_coords=p["rec_coords"])
    assert np.abs(ou).max() > 0 and np.abs(orec).max() > 0
    assert np.array_equal(u, ou)
    assert np.allclose(rec, orec, rtol=1e-12, atol=1e-12 * np.abs(orec).max())
