"""Failure detection without a GPU fault: a kernel's bounded wait on a barrier
that nothing completes gives up after its budget and says so; the device stays
usable; a timed-out or failed context reports instead of hanging."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1906_10811_b300 import build
    build.build()


def test_bounded_wait_expires_and_device_stays_usable():
    from paper_1906_10811_b300 import Solver, binding as B
    expired, waited = B.fd_selftest_bounded_wait(20.0)
    assert expired
    assert 15.0 <= waited <= 2000.0
    with Solver((20, 21, 22), (10.0,) * 3, 4, 1.0, "acoustic") as s:   # the GPU still works
        s.set_model(np.full((20, 21, 22), 0.2, np.float32))
        s.set_field(np.ones((20, 21, 22), np.float32))
        s.run(3)
        u, _ = s.read()
        assert np.isfinite(u).all()


def test_selftest_rejects_bad_budget():
    from paper_1906_10811_b300 import binding as B
    for bad in (0.0, -1.0, 1e6):
        with pytest.raises(B.FdError):
            B.fd_selftest_bounded_wait(bad)
