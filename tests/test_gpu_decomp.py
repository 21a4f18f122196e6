"""z-slab domain decomposition on one GPU, through the C ABI.

One grid cut into S = 2, 3, 4 slabs along z (each a library context with its
global placement, halos refreshed from the neighbours after every step) must
give bitwise the wavefield and traces of the unsharded run: sources sit on and
between slab interfaces, receivers straddle them, and both stream layouts
(one shared stream; a stream per slab, exchanges ordered by events) and another
tile width are covered.  The unsharded run is itself checked against the FP64
oracle.
"""

import numpy as np
import pytest

import fdsynth
from helpers import oracle_acoustic, rel_l2, small_problem

pytestmark = pytest.mark.gpu

TOL_WAVE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _problem(shape, so, nt, bounds_for):
    """Sources on the slab interfaces (on a plane, between two planes) and receivers
    straddling them, for the slab layouts in ``bounds_for``."""
    p = small_problem(shape, so, nt, nrec=20, nbl=5)
    h = p["spacing"][0]
    rng = np.random.default_rng(11)
    src, rec = [list(p["src_coords"])], [list(p["rec_coords"])]
    for bounds in bounds_for:
        for z0, _ in bounds[1:]:
            y, x = rng.uniform(6, shape[1] - 7) * h, rng.uniform(6, shape[2] - 7) * h
            src.append([np.array([z0 * h, y, x]), np.array([(z0 - 0.5) * h, y + h, x])])
            rec.append([np.array([(z0 - 0.3) * h, y + 2 * h, x - h]),
                        np.array([(z0 - 1) * h, y, x + 2 * h])])
    p["src_coords"] = np.vstack([np.vstack(s) for s in src]).astype(np.float32)
    p["rec_coords"] = np.vstack([np.vstack(r) for r in rec]).astype(np.float32)
    ns = len(p["src_coords"])
    p["wavelet"] = (np.repeat(p["wavelet"], ns, axis=1) *
                    np.linspace(0.5, 1.5, ns, dtype=np.float32)).astype(np.float32)
    return p


def _whole(p, nt, tile=None):
    import torch
    from paper_1906_10811_b300 import Solver
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", device=True) as s:
        s.set_model(dev(p["m"]), dev(p["damp"]))
        s.set_sources(dev(p["src_coords"]), dev(p["wavelet"]))
        s.set_receivers(dev(p["rec_coords"]))
        if tile:
            s.set_tile_config(**tile)
        s.run(nt)
        u, rec = s.read()
    return u.cpu().numpy(), rec.cpu().numpy()


def _slabs(p, nt, nslabs, streams="shared", tile=None, chunks=None):
    from paper_1906_10811_b300.decomp import SlabDecomposition
    with SlabDecomposition(p["shape"], p["spacing"], p["so"], p["dt"], nslabs,
                           streams=streams) as d:
        d.set_model(p["m"], p["damp"])
        d.set_sources(p["src_coords"], p["wavelet"])
        d.set_receivers(p["rec_coords"])
        if tile:
            d.set_tile_config(**tile)
        for n in (chunks or [nt]):
            d.run(n)
        u, rec = d.read()
        bounds = d.bounds
    return u.cpu().numpy(), rec.cpu().numpy(), bounds


@pytest.mark.parametrize("so", (4, 8, 16))
def test_slabs_are_bitwise_the_whole_grid(so):
    from paper_1906_10811_b300.decomp import slab_bounds
    shape, nt = (41, 38, 70), 70
    R = so // 2
    layouts = [slab_bounds(shape[0], S, R) for S in (2, 3, 4)]
    p = _problem(shape, so, nt, layouts)
    ref_u, ref_rec = _whole(p, nt)
    o = oracle_acoustic(p, nt)
    assert rel_l2(ref_u, o["u"]) <= TOL_WAVE and rel_l2(ref_rec, o["rec"]) <= TOL_WAVE
    assert np.abs(ref_rec).max() > 0
    for S in (2, 3, 4):
        u, rec, bounds = _slabs(p, nt, S)
        assert bounds == slab_bounds(shape[0], S, R)
        assert np.array_equal(u, ref_u), (so, S)
        assert np.array_equal(rec, ref_rec), (so, S)


def test_slabs_on_separate_streams_chunked_and_with_x_pair_tiles():
    shape, so, nt = (36, 40, 131), 8, 60
    from paper_1906_10811_b300.decomp import slab_bounds
    p = _problem(shape, so, nt, [slab_bounds(shape[0], 3, 4)])
    ref_u, ref_rec = _whole(p, nt)
    u, rec, _ = _slabs(p, nt, 3, streams="separate", chunks=[1, 17, 42])
    assert np.array_equal(u, ref_u) and np.array_equal(rec, ref_rec)
    # x-pair tiles with a static split, with the work queue, and 24-row tiles (12
    # consumer warps) with the queue: each slab plans its own queue over its planes
    for tile in (dict(tile_x=64, tile_y=16, aligned=1),
                 dict(tile_x=64, tile_y=16, aligned=2, ctas_per_sm=1),
                 dict(tile_x=64, tile_y=24, aligned=2)):
        u, rec, _ = _slabs(p, nt, 3, tile=tile)
        assert np.array_equal(u, ref_u) and np.array_equal(rec, ref_rec), tile


def test_halo_export_import_is_the_copy_between_slabs():
    """Two slabs stepped by hand, the halo faces moved through caller buffers
    (the route a multi-process exchange takes), match fd_run_slabs bitwise."""
    import torch
    from paper_1906_10811_b300 import binding as B
    from paper_1906_10811_b300.decomp import SlabDecomposition, SolverSlab
    shape, so, nt = (30, 33, 45), 8, 40
    p = small_problem(shape, so, nt, nrec=9, nbl=4)
    ref_u, ref_rec, _ = _slabs(p, nt, 2)
    with SlabDecomposition(shape, p["spacing"], so, p["dt"], 2) as d:
        d.set_model(p["m"], p["damp"])
        d.set_sources(p["src_coords"], p["wavelet"])
        d.set_receivers(p["rec_coords"])
        a, b = (SolverSlab(s) for s in d.slabs)
        assert a.elems == B.fd_halo_elems(d.slabs[0].ctx) > 0
        fa, fb = a.new_buffer(), b.new_buffer()
        for _ in range(nt):
            a.step()
            b.step()
            a.export_face(1, fa)
            b.export_face(0, fb)
            a.import_halo(1, fb)
            b.import_halo(0, fa)
        torch.cuda.synchronize()
        u, rec = d.read()
    assert np.array_equal(u.cpu().numpy(), ref_u) and np.array_equal(rec.cpu().numpy(), ref_rec)


def test_subdomain_calls_are_checked():
    import torch
    from paper_1906_10811_b300 import Batch, Solver
    from paper_1906_10811_b300 import binding as B
    p = small_problem((20, 24, 28), 8, 10, nrec=3)
    s = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic")
    s.set_model(p["m"], p["damp"])
    with pytest.raises(B.FdError) as e:
        B.fd_set_subdomain(s.ctx, 10, 25)          # 10 + 20 planes > 25
    assert e.value.status == B.FD_EINVAL
    s.set_receivers(p["rec_coords"])
    with pytest.raises(B.FdError) as e:
        B.fd_set_subdomain(s.ctx, 0, 40)           # after receivers
    assert e.value.status == B.FD_ESTATE
    s.close()
    s = Solver(p["shape"], p["spacing"], 8, p["dt"], "acoustic")
    s.set_model(p["m"], p["damp"])
    B.fd_set_subdomain(s.ctx, 5, 40)
    with pytest.raises(B.FdError):
        B.fd_run_slabs([s.ctx, s.ctx], 1)             # not contiguous slabs
    b = Batch(8)
    with pytest.raises(B.FdError) as e:
        b.add(s)
    assert e.value.status == B.FD_EUNSUPPORTED
    b.close()
    s.close()
    d2 = Solver((30, 40), (10.0,) * 2, 8, 0.1, "acoustic")
    with pytest.raises(B.FdError) as e:
        B.fd_set_subdomain(d2.ctx, 0, 60)
    assert e.value.status == B.FD_EUNSUPPORTED
    d2.close()
    assert torch.cuda.is_available()
