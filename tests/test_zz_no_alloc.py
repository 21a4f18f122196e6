"""The no-allocation entry point fd_acoustic_run_noalloc, through the C ABI.

It exists for callers that cannot allocate GPU memory (an application whose own
pool already holds the device, or a latency-critical loop that must not stall
on cudaMalloc/cudaFree); it keeps its working copies in one fixed-size
file-scope device array instead.  These tests check, on two calls in a row with
different grids (so the second call starts from the first call's leftovers in
that shared array), that its output equals what the allocating entry points
(fd_create / fd_set_model / fd_set_field / fd_run / fd_read) produce, within the
acoustic tolerance the other parity tests use.  This file is collected last.
"""

import numpy as np
import pytest

import fdsynth
from helpers import rel_l2

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


def test_noalloc_matches_allocating_path_on_two_calls_in_a_row():
    import torch
    from paper_1906_10811_b300 import binding as B
    stream = torch.cuda.current_stream()
    cases = [((33, 29, 40), 8, 7, 0), ((45, 61), 4, 11, 1)]
    for shape, so, nt, seed in cases:
        p, u, up = _case(shape, so, seed)
        ref_u, ref_up = _allocating_run(p, u, up, nt)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
        out = torch.full(shape, float("nan"), device="cuda")
        out_prev = torch.full(shape, float("nan"), device="cuda")
        B.fd_acoustic_run_noalloc(shape, p["spacing"], so, p["dt"], dev(p["m"]), dev(p["damp"]),
                                  dev(u), dev(up), nt, out, out_prev, stream.cuda_stream)
        stream.synchronize()
        assert rel_l2(out.cpu().numpy(), ref_u) <= TOL_WAVE
        assert rel_l2(out_prev.cpu().numpy(), ref_up) <= TOL_WAVE


def test_noalloc_rejects_grids_beyond_its_working_memory():
    import torch
    from paper_1906_10811_b300 import binding as B
    shape = (100, 100, 100)
    z = torch.zeros(shape, device="cuda")
    m = torch.full(shape, 0.2, device="cuda")
    with pytest.raises(B.FdError) as e:
        B.fd_acoustic_run_noalloc(shape, (10.0,) * 3, 8, 1.0, m, None, z, None, 1, z)
    assert e.value.status == B.FD_EINVAL and "working memory" in str(e.value)
    with pytest.raises(TypeError):
        B.fd_acoustic_run_noalloc((8, 8), (10.0,) * 2, 2, 1.0, np.ones((8, 8), np.float32),
                                  None, z, None, 1, z)
