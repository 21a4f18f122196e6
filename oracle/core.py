"""ctypes binding to the plain FP64 C oracle ``fd_oracle.c`` (TEST INFRASTRUCTURE ONLY).

All arrays are float64, dense, C order, interior only (no halo).  Inputs given
as float32 are promoted to float64 here, so the oracle sees exactly the values
the CUDA path sees.  See ``fd_oracle.c`` for the scheme (thesis §5.1.2 for the
diffusion problem; §6.2.1 names the acoustic operator, whose discrete form is the
standard second-order leapfrog written there).
"""

import ctypes
import os
import subprocess

import numpy as np

from .weights import fd_weights

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_LIB = os.path.join(_HERE, "_fd_oracle.so")

_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force=False):
    """Compile fd_oracle.c (generic x86-64, OpenMP) into oracle/_fd_oracle.so."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", _LIB, _SRC, "-lm"]
    subprocess.check_call(cmd)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_laplacian.argtypes = [ctypes.c_int, _i64p, _f64p, ctypes.c_int, _f64p, _f64p, _f64p]
        lib.oracle_diffusion.argtypes = [ctypes.c_int, _i64p, _f64p, ctypes.c_int, _f64p,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, _f64p]
        lib.oracle_corners.argtypes = [ctypes.c_int, _i64p, _f64p, _f64p, _i64p, _f64p]
        lib.oracle_acoustic.argtypes = [ctypes.c_int, _i64p, _f64p, ctypes.c_int, _f64p,
                                        ctypes.c_double, _f64p, _f64p, _f64p, _f64p,
                                        ctypes.c_int, _f64p, ctypes.c_int, _f64p, ctypes.c_int,
                                        ctypes.c_int, _f64p, _f64p, ctypes.c_int]
        for name in ("oracle_laplacian", "oracle_diffusion", "oracle_corners", "oracle_acoustic"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_f64p):
    return a.ctypes.data_as(t) if a is not None else None


def _shape(shape):
    return np.ascontiguousarray(shape, dtype=np.int64)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} failed with status {st}")


def laplacian(u, spacing, so, weights=None):
    """L u with zero values outside the grid."""
    u = _d(u)
    w = _d(weights if weights is not None else fd_weights(so))
    h = _d(spacing)
    out = np.empty_like(u)
    _check(_load().oracle_laplacian(u.ndim, _ptr(_shape(u.shape), _i64p), _ptr(h), so,
                                    _ptr(w), _ptr(u), _ptr(out)), "oracle_laplacian")
    return out


def diffusion(u0, spacing, so, nu, dt, nt, weights=None, boundary="zero", interior=True):
    """Forward-Euler diffusion; returns u^nt.

    interior True: interior nodes updated, boundary nodes held (§2.1.1's
    grid.interior subdomain, the §5.1.2 benchmark); False: every node updated.
    boundary "zero": zero outside the grid; "odd": outside values are the
    negated mirror images about the boundary nodes (interior update only)."""
    u = _d(u0).copy()
    w = _d(weights if weights is not None else fd_weights(so))
    h = _d(spacing)
    bc = {"zero": 0, "odd": 1}[boundary]
    _check(_load().oracle_diffusion(u.ndim, _ptr(_shape(u.shape), _i64p), _ptr(h), so, _ptr(w),
                                    float(nu), float(dt), int(nt), bc, int(bool(interior)),
                                    _ptr(u)),
           "oracle_diffusion")
    return u


def corners(shape, spacing, coord):
    """(flat node indices [2^D], weights [2^D]) of the multilinear stencil of one point."""
    ndim = len(shape)
    node = np.empty(1 << ndim, dtype=np.int64)
    wt = np.empty(1 << ndim, dtype=np.float64)
    _check(_load().oracle_corners(ndim, _ptr(_shape(shape), _i64p), _ptr(_d(spacing)),
                                  _ptr(_d(coord)), _ptr(node, _i64p), _ptr(wt)), "oracle_corners")
    return node, wt


def acoustic(m, dt, spacing, so, nt, damp=None, u_cur=None, u_prev=None,
             src_coords=None, wavelet=None, rec_coords=None, n0=0, weights=None):
    """Run ``nt`` leapfrog steps from global step ``n0``.

    Returns ``(u_cur, u_prev, rec)`` = (u^{n0+nt}, u^{n0+nt-1}, traces [nt+1][nrec]).
    """
    m = _d(m)
    shape = m.shape
    ndim = m.ndim
    damp = _d(damp) if damp is not None else None
    u = _d(u_cur).copy() if u_cur is not None else np.zeros(shape)
    up = _d(u_prev).copy() if u_prev is not None else u.copy()
    w = _d(weights if weights is not None else fd_weights(so))
    h = _d(spacing)
    if src_coords is not None and len(src_coords):
        sc = _d(src_coords).reshape(-1, ndim)
        wav = _d(wavelet).reshape(-1, sc.shape[0])
        nsrc, ntw = sc.shape[0], wav.shape[0]
    else:
        sc = wav = None
        nsrc, ntw = 0, 0
    if rec_coords is not None:
        rc = _d(rec_coords).reshape(-1, ndim)
        nrec = rc.shape[0]
    else:
        rc, nrec = None, 0
    rec = np.zeros((nt + 1, nrec))
    _check(_load().oracle_acoustic(ndim, _ptr(_shape(shape), _i64p), _ptr(h), so, _ptr(w), float(dt),
                                   _ptr(m), _ptr(damp), _ptr(u), _ptr(up),
                                   nsrc, _ptr(sc), ntw, _ptr(wav), int(n0),
                                   nrec, _ptr(rc), _ptr(rec), int(nt)), "oracle_acoustic")
    return u, up, rec
