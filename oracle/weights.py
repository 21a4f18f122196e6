"""Central second-derivative weights of even space order ``so`` (oracle side).

Devito's ``u.dx2`` at space order ``so`` (thesis §2.1.1, the FD shortcuts on
``TimeFunction``; §5.1.2, ``TimeFunction(..., space_order=so)`` and
``u.dx2 + u.dy2``) is the symmetric central approximation of d²/dx² on the
``2r+1`` points ``-r..r`` with ``r = so/2``.  The thesis does not print the
weights.  Here they are obtained the plain way: require the stencil to be exact
on the even monomials 1, x², x⁴, …, x^(2r) (odd ones vanish by symmetry),
which is a square linear system in ``w_0 .. w_r``; it is solved exactly in
rational arithmetic by Gaussian elimination.

Pins (tests/test_oracle_weights.py): an independent closed-form expression of
the same weights, a golden table of published values, and the observed
convergence order on smooth functions.
"""

from fractions import Fraction
from functools import lru_cache

SPACE_ORDERS = (2, 4, 6, 8, 10, 12, 14, 16)


def _solve_exact(a, b):
    """Gaussian elimination with exact Fractions; ``a`` is square, non-singular."""
    n = len(b)
    m = [list(row) + [rhs] for row, rhs in zip(a, b)]
    for col in range(n):
        piv = next(i for i in range(col, n) if m[i][col] != 0)
        m[col], m[piv] = m[piv], m[col]
        for i in range(n):
            if i != col and m[i][col] != 0:
                f = m[i][col] / m[col][col]
                m[i] = [x - f * y for x, y in zip(m[i], m[col])]
    return [m[i][n] / m[i][i] for i in range(n)]


@lru_cache(maxsize=None)
def fd_weights_fraction(so):
    """Exact weights ``(w_0, w_1, ..., w_r)`` with ``w_{-k} = w_k``.

    Moment conditions, for j = 0, 2, 4, ..., 2r:
        w_0·[j == 0] + 2·Σ_{k=1..r} w_k·k^j = 2·[j == 2]
    (the stencil applied to x^j at x = 0 must equal the exact second derivative).
    """
    if so < 2 or so % 2:
        raise ValueError("space order must be even and >= 2")
    r = so // 2
    rows, rhs = [], []
    for j in range(0, 2 * r + 1, 2):
        row = [Fraction(1 if j == 0 else 0)]
        row += [Fraction(2 * k ** j) for k in range(1, r + 1)]
        rows.append(row)
        rhs.append(Fraction(2 if j == 2 else 0))
    return tuple(_solve_exact(rows, rhs))


def fd_weights(so):
    """The exact weights rounded once to float64, as a list ``[w_0, ..., w_r]``."""
    return [float(w) for w in fd_weights_fraction(so)]
