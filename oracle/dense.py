"""Brute force on tiny grids (TEST INFRASTRUCTURE ONLY).

A second, structurally different construction of the same discrete operators,
used to pin the C oracle:

* the Laplacian is a dense matrix built as a Kronecker sum of 1-D banded
  matrices (one per axis, truncated at the grid edge = zero halo);
* the injection/interpolation operator is built from tent functions
  ``Π_d max(0, 1 - |c_d/h_d - j_d|)`` evaluated at every node, rather than
  from floor/fraction corners;
* time stepping is a plain matrix recursion.

Only for grids of a few thousand nodes.
"""

import numpy as np

from .weights import fd_weights


def second_diff_matrix(n, h, so, weights=None, odd=False):
    """1-D matrix of Σ_k w_|k| u_{i+k} / h² with zero outside 0..n-1, or with
    ``odd``: a column i+k outside the grid folds onto its mirror node about the
    boundary node (0 or n-1) with the weight negated."""
    w = weights if weights is not None else fd_weights(so)
    r = so // 2
    a = np.zeros((n, n))
    for i in range(n):
        for k in range(-r, r + 1):
            j = i + k
            if 0 <= j < n:
                a[i, j] += w[abs(k)] / (h * h)
            elif odd:
                jm = -j if j < 0 else 2 * (n - 1) - j
                a[i, jm] -= w[abs(k)] / (h * h)
    return a


def laplacian_matrix(shape, spacing, so, weights=None, odd=False):
    """Kronecker sum over axes; row-major (C order) flattening."""
    mats = [second_diff_matrix(n, h, so, weights, odd) for n, h in zip(shape, spacing)]
    size = int(np.prod(shape))
    lap = np.zeros((size, size))
    for d, md in enumerate(mats):
        term = np.ones((1, 1))
        for e, n in enumerate(shape):
            term = np.kron(term, md if e == d else np.eye(n))
        lap += term
    return lap


def tent_row(shape, spacing, coord):
    """Interpolation weights of one point at every node (dense row)."""
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    wt = np.ones(shape)
    for d, g in enumerate(grids):
        wt = wt * np.maximum(0.0, 1.0 - np.abs(coord[d] / spacing[d] - g))
    return wt.reshape(-1)


def diffusion(u0, spacing, so, nu, dt, nt, weights=None, boundary="zero", interior_only=True):
    shape = u0.shape
    lap = laplacian_matrix(shape, spacing, so, weights, odd=boundary == "odd")
    interior = np.ones(shape, dtype=bool)
    for d, n in enumerate(shape):
        if not interior_only:
            break
        sl = [slice(None)] * len(shape)
        sl[d] = 0
        interior[tuple(sl)] = False
        sl[d] = n - 1
        interior[tuple(sl)] = False
    mask = interior.reshape(-1).astype(np.float64)
    step = np.eye(lap.shape[0]) + nu * dt * (mask[:, None] * lap)
    u = u0.reshape(-1).astype(np.float64)
    for _ in range(nt):
        u = step @ u
    return u.reshape(shape)


def acoustic(m, dt, spacing, so, nt, damp=None, u_cur=None, u_prev=None,
             src_coords=None, wavelet=None, rec_coords=None, n0=0, weights=None):
    shape = m.shape
    mm = m.reshape(-1).astype(np.float64)
    sig = (damp.reshape(-1).astype(np.float64) if damp is not None else np.zeros_like(mm)) * dt / 2
    lap = laplacian_matrix(shape, spacing, so, weights)
    u = (u_cur.reshape(-1).astype(np.float64) if u_cur is not None else np.zeros_like(mm))
    up = (u_prev.reshape(-1).astype(np.float64) if u_prev is not None else u.copy())
    ps = np.array([tent_row(shape, spacing, c) for c in src_coords]) if src_coords is not None and len(src_coords) else None
    pr = np.array([tent_row(shape, spacing, c) for c in rec_coords]) if rec_coords is not None else None
    traces = [pr @ u] if pr is not None else []
    for s in range(nt):
        un = (dt * dt * (lap @ u) + 2 * mm * u - (mm - sig) * up) / (mm + sig)
        if ps is not None:
            un = un + (ps.T @ np.asarray(wavelet, dtype=np.float64)[n0 + s]) * dt * dt / mm
        up, u = u, un
        if pr is not None:
            traces.append(pr @ u)
    rec = np.array(traces) if pr is not None else None
    return u.reshape(shape), up.reshape(shape), rec
