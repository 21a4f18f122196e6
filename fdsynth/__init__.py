"""Seeded synthetic inputs for the finite-difference sweep.

This module only *generates problem data* (initial fields, velocity models,
damping profiles, wavelets, coordinates, time steps).  It holds none of the
scheme's arithmetic: no stencil weights, no time update, no injection or
interpolation.  Both the CUDA path and the oracle consume the arrays it
returns, as float32, so that a parity test measures arithmetic only.

Axis convention everywhere: C order, axis 0 slowest.  In 3D axis 0 is depth
(z), axis 2 is x (contiguous).  Coordinates are given per axis in the same
order as the shape.  Units for the acoustic problems: metres, milliseconds,
km/s (= m/ms) and kHz, so ``m = 1/v²`` in ms²/m².
"""

import math

import numpy as np


def f32(x):
    """Round a Python/numpy float to the nearest float32 and return it as float."""
    return float(np.float32(x))


# --------------------------------------------------------------------------
# Diffusion (thesis §5.1.2: u_t = ν (u_xx + u_yy), time order 1)
# --------------------------------------------------------------------------

def diffusion_problem(n=128, ndim=2, nu=0.5, courant=0.2, mode=(1, 1, 1)):
    """Sine-mode initial data on [0,1]^ndim with n nodes per axis (boundary included).

    Spacing h = 1/(n-1) (nodes at i*h, both ends on the boundary); dt chosen so
    that ν dt / h² = ``courant`` (0.2 gives dt = 0.2 h²/0.5 for ν = 0.5).
    u0 = Π_d sin(k_d π x_d), evaluated in float64, boundary nodes set to exactly
    0, rounded once to float32.
    Returns dict(u0, spacing, dt, nu).
    """
    h = 1.0 / (n - 1)
    x = np.arange(n, dtype=np.float64) * h
    u = np.ones((1,) * 0)
    for d in range(ndim):
        s = np.sin(mode[d] * math.pi * x)
        s[0] = 0.0
        s[-1] = 0.0
        u = np.multiply.outer(u, s) if u.ndim else s
    dt = f32(courant * h * h / nu)
    return dict(u0=u.astype(np.float32), spacing=(h,) * ndim, dt=dt, nu=nu)


def random_field(shape, seed=0, scale=1.0):
    """Uniform(-scale, scale) float32 field."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-scale, scale, size=shape)).astype(np.float32)


# --------------------------------------------------------------------------
# Acoustic model recipe
# --------------------------------------------------------------------------

def _gaussian_smooth(a, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sigma, mode="reflect")


def velocity_model(shape, seed=0, vmin=1.5, vmax=4.5, nlayers=6, noise=0.05,
                   smooth=3.0, clip=(1.4, 4.8)):
    """Layered velocity (km/s) along axis 0 with smoothed Gaussian noise.

    ``nlayers`` bands with interfaces at sorted uniform depths; band velocities
    sorted uniform in [vmin, vmax] with the first = vmin and the last = vmax;
    times (1 + noise·n), n = white Gaussian noise smoothed by a Gaussian filter
    (σ = ``smooth`` cells) and renormalised to unit std; clipped to ``clip``.
    Computed in float64, rounded once to float32.
    """
    rng = np.random.default_rng(seed)
    nz = shape[0]
    cuts = np.sort(rng.uniform(0, nz, size=nlayers - 1))
    vel = np.sort(rng.uniform(vmin, vmax, size=nlayers))
    vel[0], vel[-1] = vmin, vmax
    band = np.searchsorted(cuts, np.arange(nz) + 0.5)
    v1 = vel[band]
    v = np.broadcast_to(v1.reshape((nz,) + (1,) * (len(shape) - 1)), shape).astype(np.float64)
    if noise:
        nrng = np.random.default_rng(seed + 1)
        nz_field = nrng.standard_normal(shape)
        nz_field = _gaussian_smooth(nz_field, smooth)
        nz_field /= nz_field.std()
        v = v * (1.0 + noise * nz_field)
    v = np.clip(v, clip[0], clip[1])
    return v.astype(np.float32)


def slowness_squared(v):
    """m = 1/v² in float64 from float32 v, rounded to float32."""
    return (1.0 / (v.astype(np.float64) ** 2)).astype(np.float32)


def damping_profile(shape, spacing, v, nbl=40, R=1e-3):
    """Absorbing-layer coefficient ``damp`` (float32), zero in the interior.

    s_d ∈ (0, 1] is the normalised depth into the layer along axis d (0 outside
    it); damp = m · σ_max · Σ_d (s_d − sin(2π s_d)/(2π)),
    σ_max = 2 v_max ln(1/R) / (nbl h).
    """
    m = 1.0 / (v.astype(np.float64) ** 2)
    vmax = float(np.max(v))
    prof = np.zeros(shape)
    for d, n in enumerate(shape):
        h = spacing[d]
        smax = 2.0 * vmax * math.log(1.0 / R) / (nbl * h)
        i = np.arange(n, dtype=np.float64)
        s = np.zeros(n)
        lo = i < nbl
        hi = i > n - 1 - nbl
        s[lo] = (nbl - i[lo]) / nbl
        s[hi] = (i[hi] - (n - 1 - nbl)) / nbl
        p = smax * (s - np.sin(2 * math.pi * s) / (2 * math.pi))
        p[~(lo | hi)] = 0.0
        prof = prof + p.reshape([n if e == d else 1 for e in range(len(shape))])
    return (m * prof).astype(np.float32)


def cfl_dt(v, h, ndim, c=None):
    """dt = c·h/max(v), c = 0.38 (3D) or 0.42 (2D), rounded to float32."""
    if c is None:
        c = 0.38 if ndim == 3 else 0.42
    return f32(c * h / float(np.max(v)))


def ricker(nt, dt, f0=0.010, t0=None):
    """Ricker wavelet s(t_n), t_n = n·dt, t0 = 1/f0; float64 libm, then float32."""
    if t0 is None:
        t0 = 1.0 / f0
    t = np.arange(nt, dtype=np.float64) * dt
    a = (math.pi * f0 * (t - t0)) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float32)


def centre(shape, spacing):
    """Physical coordinates of the domain centre ((n-1)h/2 per axis), float32."""
    return np.array([(n - 1) * h / 2.0 for n, h in zip(shape, spacing)], dtype=np.float32)


def receiver_line(shape, spacing, nrec, nbl, depth_offset=5):
    """``nrec`` receivers along the last axis spanning the physical interior.

    Other axes: centre, except axis 0 (depth) at the centre + ``depth_offset``
    cells.  Returns float32 [nrec][ndim].
    """
    ndim = len(shape)
    c = centre(shape, spacing).astype(np.float64)
    out = np.empty((nrec, ndim))
    for d in range(ndim):
        out[:, d] = c[d]
    out[:, 0] = c[0] + depth_offset * spacing[0]
    nx, hx = shape[-1], spacing[-1]
    lo, hi = nbl * hx, (nx - 1 - nbl) * hx
    out[:, -1] = np.linspace(lo, hi, nrec) if nrec > 1 else (lo + hi) / 2
    return out.astype(np.float32)


def random_points(shape, spacing, npts, seed=0, margin=0.0):
    """Uniform random coordinates inside the grid (float32 [npts][ndim])."""
    rng = np.random.default_rng(seed)
    out = np.empty((npts, len(shape)))
    for d, (n, h) in enumerate(zip(shape, spacing)):
        out[:, d] = rng.uniform(margin * h, (n - 1 - margin) * h, size=npts)
    return out.astype(np.float32)


def acoustic_problem(n=256, ndim=3, so=8, nbl=40, h=10.0, nt=500, nrec=256,
                     seed=0, f0=0.010, noise=0.05, vel=None):
    """The layered acoustic shot: m, damp, dt, one centred Ricker source, a receiver line.

    ``n`` is the full grid (damping layer inside it).  Returns a dict with float32
    arrays and float32-representable scalars.
    """
    shape = (n,) * ndim if np.isscalar(n) else tuple(n)
    spacing = (float(h),) * ndim
    v = vel if vel is not None else velocity_model(shape, seed=seed, noise=noise)
    m = slowness_squared(v)
    damp = damping_profile(shape, spacing, v, nbl=nbl)
    dt = cfl_dt(v, h, ndim)
    src = centre(shape, spacing).reshape(1, ndim)
    wav = ricker(nt, dt, f0).reshape(nt, 1)
    rec = receiver_line(shape, spacing, nrec, nbl) if nrec else np.zeros((0, ndim), np.float32)
    return dict(shape=shape, spacing=spacing, so=so, dt=dt, nt=nt, m=m, damp=damp,
                vel=v, src_coords=src, wavelet=wav, rec_coords=rec)


def perturbed_model(m, nbl, seed=3, amp=0.05, nblobs=4, width=0.08):
    """A seeded "true" model for inversion: m·(1 + amp·Σ_b exp(−|x − c_b|²/(2 s²))).

    ``nblobs`` Gaussian blobs with centres uniform inside the region the
    damping layer leaves (``nbl`` cells from every face) and width s =
    ``width``·(smallest extent).  m only grows (the velocity only drops), so a
    dt stable for m stays stable.  Float64, rounded once to float32.
    """
    shape = m.shape
    rng = np.random.default_rng(seed)
    s = width * min(shape)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij",
                        sparse=True)
    bump = np.zeros(shape)
    for _ in range(nblobs):
        c = [rng.uniform(min(nbl, n // 4), max(n - 1 - nbl, n - 1 - n // 4)) for n in shape]
        r2 = sum((g - cc) ** 2 for g, cc in zip(grids, c))
        bump += np.exp(-r2 / (2.0 * s * s))
    return (m.astype(np.float64) * (1.0 + amp * bump)).astype(np.float32)


def serving_stream(nshots=64, seed=2, mean_gap_s=0.01, sizes2d=(200, 1000), sizes3d=(128, 320),
                   nt_range=(300, 1000), nrec_range=(128, 512), so=8, frac3d=0.5, nbl=40):
    """A seeded Poisson stream of acoustic shots for the serving workload.

    Each shot: a 2-D grid of n² (n uniform in ``sizes2d``) or a 3-D grid of n³
    (n uniform in ``sizes3d``), chosen with probability ``frac3d``; the layered
    model recipe with its own seed; one Ricker source at the centre; a receiver
    line of nrec (uniform in ``nrec_range``) receivers; nt uniform in
    ``nt_range`` steps.  Arrival gaps are exponential with mean ``mean_gap_s``.
    Returns a list of (id, arrival seconds, problem dict).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(nshots):
        t += float(rng.exponential(mean_gap_s))
        three = bool(rng.random() < frac3d)
        lo, hi = sizes3d if three else sizes2d
        n = int(rng.integers(lo, hi + 1))
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        nrec = int(rng.integers(nrec_range[0], nrec_range[1] + 1))
        layer = min(nbl, max(4, n // 8))
        p = acoustic_problem(n=n, ndim=3 if three else 2, so=so, nbl=layer, nt=nt, nrec=nrec,
                             seed=1000 + i)
        out.append((i, t, p))
    return out
