"""Shared helpers for the GPU parity tests (comparison metrics, run wrappers)."""

import numpy as np

import fdsynth
from oracle import core as oracle


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def gpu_acoustic(p, nt, kernel="auto", graphs=True, profile=False, device=False, damp=True,
                 with_src=True, with_rec=True, chunks=None, tile=None):
    """Run a problem dict from fdsynth.acoustic_problem through the C ABI.

    tile: a tile configuration for the pipelined kernel (Solver.set_tile_config
    keywords), set once sources and receivers are in place."""
    from paper_1906_10811_b300 import Solver
    s = Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", kernel=kernel,
               graphs=graphs, profile=profile, device=device)
    conv = _to_device if device else (lambda x: x)
    s.set_model(conv(p["m"]), conv(p["damp"]) if damp else None)
    if with_src:
        s.set_sources(conv(p["src_coords"]), conv(p["wavelet"]))
    if with_rec:
        s.set_receivers(conv(p["rec_coords"]))
    if tile is not None:
        s.set_tile_config(**tile)
    used = s.tile_config if s.kernel_name.startswith("stencil3d_") and \
        s.kernel_name != "stencil3d_plain" else None
    for n in (chunks or [nt]):
        s.run(n)
    u, rec = s.read()
    up = s.read_prev()
    name = s.kernel_name
    prof = s.profile() if profile else None
    s.close()
    if device:
        u, up = u.cpu().numpy(), up.cpu().numpy()
        rec = rec.cpu().numpy() if rec is not None else None
    return dict(u=u, u_prev=up, rec=rec, kernel=name, profile=prof, tile=used)


def oracle_acoustic(p, nt, damp=True, with_src=True, with_rec=True):
    u, up, rec = oracle.acoustic(p["m"], p["dt"], p["spacing"], p["so"], nt,
                                 damp=p["damp"] if damp else None,
                                 src_coords=p["src_coords"] if with_src else None,
                                 wavelet=p["wavelet"] if with_src else None,
                                 rec_coords=p["rec_coords"] if with_rec else None)
    return dict(u=u, u_prev=up, rec=rec)


def _to_device(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def small_problem(shape, so, nt, nrec=12, nbl=6, seed=0):
    return fdsynth.acoustic_problem(n=shape, ndim=len(shape), so=so, nbl=nbl, nt=nt, nrec=nrec,
                                    seed=seed, f0=0.03)
