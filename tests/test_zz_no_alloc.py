"""The no-allocation entry point fd_acoustic_run_noalloc, through the C ABI.

Some callers cannot allocate GPU memory: an application whose own memory pool
already holds the device (a cudaMalloc would fail, or would go around the
pool's accounting), or a latency-critical loop that must not stall on
cudaMalloc/cudaFree.  For them the library keeps its working copies in one
fixed-size file-scope device array instead of allocating.

These tests make two calls in a row with different grids, so the second call
starts from whatever the first one left in that shared array, and check each
against the allocating entry points (fd_create / fd_set_model / fd_set_field /
fd_run / fd_read with the plain kernel, the same kernel and coefficients, so
bitwise equal) and against the FP64 oracle at the acoustic tolerance the other
parity tests use.  This file is collected last.
"""

import numpy as np
import pytest

import fdsynth
from helpers import rel_l2
from oracle import core as oracle

pytestmark = pytest.mark.gpu

TOL_WAVE = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def _case(shape, so, seed):
    p = fdsynth.acoustic_problem(n=shape, ndim=len(shape), so=so, nbl=5, nt=1, nrec=0, seed=seed)
    u = fdsynth.random_field(shape, seed=seed + 10)
    up = fdsynth.random_field(shape, seed=seed + 20)
    return p, u, up


def _allocating_run(p, u, up, nt):
    from paper_1906_10811_b300 import Solver
    with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", kernel="plain") as s:
        s.set_model(p["m"], p["damp"])
        s.set_field(u, up)
        s.run(nt)
        out, _ = s.read(traces=False)
        prev = s.read_prev()
    return out, prev


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    import torch
    from paper_1906_10811_b300 import binding as B
    stream = torch.cuda.current_stream()
    cases = [((33, 29, 40), 8, 7, 0), ((45, 61), 4, 11, 1)]
    for shape, so, nt, seed in cases:
        p, u, up = _case(shape, so, seed)
        ref_u, ref_up = _allocating_run(p, u, up, nt)
        out = torch.full(shape, float("nan"), device="cuda")
        out_prev = torch.full(shape, float("nan"), device="cuda")
        B.fd_acoustic_run_noalloc(shape, p["spacing"], so, p["dt"], _dev(p["m"]), _dev(p["damp"]),
                                  _dev(u), _dev(up), nt, out, out_prev, stream)
        stream.synchronize()
        got_u, got_up = out.cpu().numpy(), out_prev.cpu().numpy()
        # same kernel, same coefficients: bitwise the allocating path
        assert np.array_equal(got_u, ref_u)
        assert np.array_equal(got_up, ref_up)
        ou, oup, _ = oracle.acoustic(p["m"], p["dt"], p["spacing"], so, nt, damp=p["damp"],
                                     u_cur=u, u_prev=up)
        assert rel_l2(got_u, ou) <= TOL_WAVE
        assert rel_l2(got_up, oup) <= TOL_WAVE


def test_noalloc_rejects_grids_beyond_its_working_memory():
    import torch
    from paper_1906_10811_b300 import binding as B
    shape = (100, 100, 100)
    z = torch.zeros(shape, device="cuda")
    m = torch.full(shape, 0.2, device="cuda")
    with pytest.raises(B.FdError) as e:
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 3, 8, 1.0, m, None, z, None, 1, z)
    assert e.value.status == B.FD_EINVAL and "working memory" in str(e.value)


def test_noalloc_rejects_arrays_it_cannot_use_before_calling_the_library():
    import torch
    from paper_1906_10811_b300 import binding as B
    shape = (8, 9)
    m = torch.full(shape, 0.2, device="cuda")
    z = torch.zeros(shape, device="cuda")
    small = torch.zeros(8 * 9 - 1, device="cuda")
    with pytest.raises(TypeError):           # host array
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 2, 2, 1.0, np.ones(shape, np.float32),
                                  None, z, None, 1, z)
    with pytest.raises(ValueError):          # too few elements: would be read out of bounds
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 2, 2, 1.0, m, None, small, None, 1, z)
    with pytest.raises(ValueError):          # output too small: would be written out of bounds
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 2, 2, 1.0, m, None, z, None, 1, small)
    with pytest.raises(TypeError):           # wrong dtype
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 2, 2, 1.0, m.double(), None, z, None, 1, z)
    with pytest.raises(TypeError):           # not contiguous
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 2, 2, 1.0, m, None,
                                  torch.zeros((9, 8), device="cuda").t(), None, 1, z)
