"""FP64 FWI objective and gradient (TEST INFRASTRUCTURE ONLY).

Objective: J(m) = ½ Σ_{n=0..N} ||P_r u^n(m) − d^n||² for the acoustic leapfrog
of ``fd_oracle.c`` (u^0 = u^{-1} = 0, damp independent of m).

Gradient by the adjoint-state method of the discrete scheme.  Writing the
update as u^{n+1} = a·L u^n + b·u^n − c·u^{n−1} + q_n with D = m+σ,
a = dt²/D, b = 2m/D, c = (m−σ)/D and q_n = P_sᵀ(dt² s_n / m), the adjoint
variable ν = a·λ (λ the Lagrange multipliers of the updates) obeys the
forward recursion run backwards,

    ν^k = a·L ν^{k+1} + b·ν^{k+1} − c·ν^{k+2} + a·P_rᵀ r^k,   k = N..1,
    ν^{N+1} = ν^{N+2} = 0,   r^k = P_r u^k − d^k,

and dJ/dm = Σ_n λ^{n+1}·∂F_n/∂m reduces to

    g = −(1/dt²) Σ_{n=0}^{N−1} ν^{n+1} ⊙ (u^{n+1} − 2u^n + u^{n−1})
        − Σ_{n=0}^{N−1} ν^{n+1} ⊙ P_sᵀ(w s_n σ / m²)          (zero where σ = 0).

Pinned by central finite differences of J on tiny grids (tests/test_oracle_fwi.py).
Everything is float64 and stores every time level (small grids only).
"""

import numpy as np

from . import core
from .weights import fd_weights


def _corner_matrix(shape, spacing, coords):
    """Dense [npoints][N] matrix of multilinear weights (rows: points)."""
    n = int(np.prod(shape))
    P = np.zeros((len(coords), n))
    for i, c in enumerate(coords):
        node, wt = core.corners(shape, spacing, c)
        np.add.at(P[i], node, wt)
    return P


def forward_states(m, damp, dt, spacing, so, nt, src_coords, wavelet):
    """All levels u^{-1}, u^0, ..., u^N (float64, [N+2][...])."""
    m = np.asarray(m, np.float64)
    shape = m.shape
    states = [np.zeros(shape), np.zeros(shape)]
    u, up = states[1], states[0]
    for n in range(nt):
        u2, u1, _ = core.acoustic(m, dt, spacing, so, 1, damp=damp, u_cur=u, u_prev=up,
                                  src_coords=src_coords, wavelet=wavelet, n0=n)
        states.append(u2)
        up, u = u, u2
    return np.array(states)


def objective(m, damp, dt, spacing, so, nt, src_coords, wavelet, rec_coords, d_obs):
    m = np.asarray(m, np.float64)
    _, _, rec = core.acoustic(m, dt, spacing, so, nt, damp=damp, src_coords=src_coords,
                              wavelet=wavelet, rec_coords=rec_coords)
    r = rec - np.asarray(d_obs, np.float64)
    return 0.5 * float(np.sum(r * r)), rec


def gradient(m, damp, dt, spacing, so, nt, src_coords, wavelet, rec_coords, d_obs):
    """(J, dJ/dm) in float64."""
    m = np.asarray(m, np.float64)
    shape = m.shape
    damp = np.zeros(shape) if damp is None else np.asarray(damp, np.float64)
    w = fd_weights(so)
    sig = damp * dt / 2.0
    D = m + sig
    a, b, c = dt * dt / D, 2 * m / D, (m - sig) / D
    U = forward_states(m, damp, dt, spacing, so, nt, src_coords, wavelet)   # U[n+1] = u^n
    Pr = _corner_matrix(shape, spacing, rec_coords)
    Ps = _corner_matrix(shape, spacing, src_coords)
    rec = np.array([Pr @ U[n + 1].reshape(-1) for n in range(nt + 1)])
    r = rec - np.asarray(d_obs, np.float64)
    J = 0.5 * float(np.sum(r * r))
    s = np.asarray(wavelet, np.float64).reshape(-1, len(src_coords))
    nu_next = np.zeros(shape)       # ν^{k+1}
    nu_next2 = np.zeros(shape)      # ν^{k+2}
    g = np.zeros(shape)
    for k in range(nt, 0, -1):
        lap = core.laplacian(nu_next, spacing, so, w)
        nu = a * lap + b * nu_next - c * nu_next2 + a * (Pr.T @ r[k]).reshape(shape)
        n = k - 1                   # ν^{n+1} = ν^k meets the update of step n
        d2u = U[n + 2] - 2 * U[n + 1] + U[n]
        g -= nu * d2u / (dt * dt)
        g -= nu * (Ps.T @ s[n]).reshape(shape) * sig / (m * m)
        nu_next2, nu_next = nu_next, nu
    return J, g
