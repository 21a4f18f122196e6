"""Pins for the oracle's finite-difference weights (Devito's ``u.dx2`` at space
order so, thesis §2.1.1 / §5.1.2).  Nothing here re-types the moment system the
oracle solves: the weights are checked against an independent closed form, a
published table and their observed convergence order."""

import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import core
from oracle.weights import SPACE_ORDERS, fd_weights, fd_weights_fraction

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fd_weights_published.txt")


def _closed_form(so):
    """w_k = 2 (-1)^(k+1) (r!)² / (k² (r-k)! (r+k)!),  w_0 = -2 Σ_k w_k."""
    r = so // 2
    wk = [Fraction(2 * (-1) ** (k + 1) * math.factorial(r) ** 2,
                   k * k * math.factorial(r - k) * math.factorial(r + k)) for k in range(1, r + 1)]
    return tuple([-2 * sum(wk)] + wk)


@pytest.mark.parametrize("so", SPACE_ORDERS)
def test_weights_match_closed_form(so):
    assert fd_weights_fraction(so) == _closed_form(so)


def test_weights_match_published_table():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for row in rows:
        so = int(row[0])
        assert fd_weights_fraction(so) == tuple(Fraction(x) for x in row[1:])


@pytest.mark.parametrize("so", SPACE_ORDERS)
def test_weights_reproduce_parabola_and_annihilate_constants(so):
    w = fd_weights_fraction(so)
    r = so // 2
    assert w[0] + 2 * sum(w[1:]) == 0                              # constants
    assert sum(w[abs(k)] * Fraction(k) ** 2 for k in range(-r, r + 1)) == 2  # x² -> 2
    # an independent exactness check: (x+1/3)^(so+1) has an exact 2nd derivative
    p = lambda x: (Fraction(x) + Fraction(1, 3)) ** (so + 1)
    d2 = (so + 1) * so * Fraction(1, 3) ** (so - 1)
    assert sum(w[abs(k)] * p(k) for k in range(-r, r + 1)) == d2


def test_bad_space_order_rejected():
    for so in (0, 1, 3, -2):
        with pytest.raises(ValueError):
            fd_weights_fraction(so)


@pytest.mark.parametrize("so", (2, 4, 6, 8))
@pytest.mark.parametrize("ndim", (2, 3))
def test_laplacian_convergence_order(so, ndim):
    """error of the oracle's L on a smooth function scales as h^so."""
    kx = (2.3, 1.7, 2.9)[:ndim]
    errs = []
    for n in (16, 32):
        h = 2.0 / (n - 1)
        g = np.meshgrid(*[np.arange(n) * h for _ in range(ndim)], indexing="ij")
        f = np.sin(sum(k * x for k, x in zip(kx, g)) + 0.3)
        exact = -sum(k * k for k in kx) * f
        lap = core.laplacian(f, (h,) * ndim, so)
        box = np.ones(f.shape, dtype=bool)      # a fixed physical box inside the grid
        for x in g:
            box &= (x > 0.6) & (x < 1.4)
        errs.append(np.abs(lap - exact)[box].max())
    order = math.log(errs[0] / errs[1]) / math.log(31 / 15)
    assert abs(order - so) < 0.1, (errs, order)


def test_symbol_at_nyquist():
    """S_so = -(w_0 + 2 Σ (-1)^k w_k): the largest eigenvalue magnitude of the 1-D
    stencil (times h²), which sets the stability limits.  S_2 = 4 and S_4 = 16/3
    follow by hand; the rest must increase monotonically below π² (the continuum
    value the sequence approaches)."""
    s = []
    for so in SPACE_ORDERS:
        w = fd_weights_fraction(so)
        s.append(-(w[0] + 2 * sum((-1) ** k * w[k] for k in range(1, len(w)))))
    assert s[0] == 4 and s[1] == Fraction(16, 3)
    assert all(a < b for a, b in zip(s, s[1:])) and float(s[-1]) < math.pi ** 2
