"""Host-side checks of the C ABI (no GPU): the library loads and exports every
symbol include/fd.h declares; host-only helpers agree with the oracle; argument
validation answers FD_EINVAL before touching the GPU; the product path fails
loudly when the library is missing."""

import ctypes
import math
import os
import re

import pytest

from oracle.weights import SPACE_ORDERS, fd_weights as oracle_weights

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1906_10811_b300 import binding, build
    build.build()
    return binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fd_create", "fd_set_model", "fd_set_sources", "fd_set_receivers",
                     "fd_run", "fd_read", "fd_destroy", "fd_last_error", "fd_set_field"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1906_10811_b300 import binding
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, f"binding lacks {name}"


def test_weights_match_oracle(lib):
    from paper_1906_10811_b300 import fd_weights
    for so in SPACE_ORDERS:
        a, b = fd_weights(so), oracle_weights(so)
        assert len(a) == len(b)
        for x, y in zip(a, b):
            assert abs(x - y) <= 1e-15 * max(1.0, abs(y))


def test_stability_symbol(lib):
    from paper_1906_10811_b300 import fd_stability_symbol
    assert abs(fd_stability_symbol(2) - 4.0) < 1e-14
    assert abs(fd_stability_symbol(4) - 16.0 / 3.0) < 1e-14
    assert math.isnan(fd_stability_symbol(5))
    vals = [fd_stability_symbol(so) for so in SPACE_ORDERS]
    assert all(a < b for a, b in zip(vals, vals[1:])) and vals[-1] < math.pi ** 2


def test_bad_orders_rejected(lib):
    from paper_1906_10811_b300 import FdError, fd_weights
    for so in (0, 1, 3, 18, -2):
        with pytest.raises(FdError):
            fd_weights(so)


def test_options_default(lib):
    from paper_1906_10811_b300 import fd_options_default
    o = fd_options_default()
    assert o.nu == 0.5 and o.use_graphs == 1 and o.device_ptrs == 0 and o.profile == 0
    assert o.kernel == 0 and o.cuda_stream is None
    assert o.dirichlet_interior == 1           # the §5.1.2 benchmark's interior update


@pytest.mark.parametrize("args,msg", [
    ((4, (8, 8, 8, 8), (1.0,) * 4, 4, 0.1, 1), "ndim"),
    ((3, (8, 8, 8), (1.0, 1.0, 1.0), 3, 0.1, 1), "space_order"),
    ((3, (8, 8, 8), (1.0, 1.0, 1.0), 18, 0.1, 1), "space_order"),
    ((3, (8, 1, 8), (1.0, 1.0, 1.0), 4, 0.1, 1), "shape"),
    ((2, (0, 8), (1.0, 1.0), 4, 0.1, 0), "shape"),
    ((3, (8, 8, 8), (1.0, -1.0, 1.0), 4, 0.1, 1), "spacing"),
    ((3, (8, 8, 8), (1.0, 1.0, 1.0), 4, 0.0, 1), "dt"),
    ((3, (8, 8, 8), (1.0, 1.0, 1.0), 4, float("nan"), 1), "dt"),
    ((2, (8, 8), (1.0, 1.0), 4, 0.1, 7), "equation"),
    # diffusion, so=2: nu dt (4/h^2 + 4/h^2) = 0.5 * 0.6 * 8 = 2.4 > 2
    ((2, (8, 8), (1.0, 1.0), 2, 0.6, 0), "forward-Euler"),
])
def test_create_validation(lib, args, msg):
    from paper_1906_10811_b300 import FdError, fd_create, binding
    with pytest.raises(FdError) as ei:
        fd_create(*args)
    assert ei.value.status == binding.FD_EINVAL
    assert msg in str(ei.value)


def test_create_at_the_diffusion_limit_passes_validation(lib):
    """exactly at ν dt Σ S/h² = 2 the arguments are valid; without a GPU the
    call then fails on the device, not on validation."""
    from paper_1906_10811_b300 import FdError, fd_create, binding
    try:
        ctx = fd_create(2, (8, 8), (1.0, 1.0), 2, 0.5, 0)
    except FdError as e:
        assert e.status in (binding.FD_ECUDA, binding.FD_ENOMEM)
    else:
        binding.fd_destroy(ctx)


def test_null_context_calls_are_safe(lib):
    assert lib.fd_steps_done(None) == -1
    assert lib.fd_run(None, 1) == 1
    lib.fd_destroy(None)
    assert lib.fd_kernel_name(None) == b"none"


def test_missing_library_fails_loudly(tmp_path):
    from paper_1906_10811_b300 import binding
    with pytest.raises(OSError):
        binding.load(str(tmp_path / "libfd_b300.so"))
