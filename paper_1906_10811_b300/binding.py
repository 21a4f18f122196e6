"""Thin ctypes binding of the C ABI in include/fd.h (argument marshalling only).

Every function keeps the C name and meaning.  Arrays may be numpy arrays (host)
or torch CUDA tensors (device; the context must then be created with
``device_ptrs=1``); they must be float32 and C-contiguous, or they are
converted.  Statuses other than FD_OK raise :class:`FdError` carrying the
status and ``fd_last_error``.  There is no fallback: if the CUDA library is
missing, loading fails loudly.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfd_b300.so")

FD_OK, FD_EINVAL, FD_ENOMEM, FD_ECUDA, FD_ESTATE, FD_ETIMEOUT, FD_EUNSUPPORTED = range(7)
STATUS_NAMES = ["FD_OK", "FD_EINVAL", "FD_ENOMEM", "FD_ECUDA", "FD_ESTATE", "FD_ETIMEOUT",
                "FD_EUNSUPPORTED"]
FD_DIFFUSION, FD_ACOUSTIC = 0, 1
FD_KERNEL_AUTO, FD_KERNEL_PLAIN, FD_KERNEL_TMA = 0, 1, 2
FD_BOUNDARY_ZERO, FD_BOUNDARY_ODD = 0, 1


class FdError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class fd_options(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("device_ptrs", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("profile", ctypes.c_int), ("kernel", ctypes.c_int),
                ("autotune", ctypes.c_int), ("boundary", ctypes.c_int),
                ("dirichlet_interior", ctypes.c_int)]


class fd_tile_config(ctypes.Structure):
    _fields_ = [("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("zblock", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("aligned", ctypes.c_int),
                ("skip_c", ctypes.c_int), ("us_per_step", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64

# name -> (restype, argtypes); every entry point declared in include/fd.h
SIGNATURES = {
    "fd_options_default": (None, [ctypes.POINTER(fd_options)]),
    "fd_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_i64),
                                 ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.POINTER(fd_options)]),
    "fd_set_model": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_set_field": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_set_sources": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, _vp]),
    "fd_set_receivers": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "fd_run": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_read": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_read_prev": (ctypes.c_int, [_vp, _vp]),
    "fd_set_step": (ctypes.c_int, [_vp, _i64]),
    "fd_reset": (ctypes.c_int, [_vp]),
    "fd_steps_done": (_i64, [_vp]),
    "fd_profile": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)]),
    "fd_kernel_name": (ctypes.c_char_p, [_vp]),
    "fd_skip_c_planes": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "fd_set_subdomain": (ctypes.c_int, [_vp, _i64, _i64]),
    "fd_halo_elems": (_i64, [_vp]),
    "fd_halo_copy": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "fd_halo_export": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "fd_halo_import": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "fd_run_slabs": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int]),
    "fd_accumulate_traces": (ctypes.c_int, [_vp, _vp]),
    "fd_get_tile_config": (ctypes.c_int, [_vp, ctypes.POINTER(fd_tile_config)]),
    "fd_set_tile_config": (ctypes.c_int, [_vp, ctypes.POINTER(fd_tile_config)]),
    "fd_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(fd_tile_config),
                                   ctypes.POINTER(fd_tile_config), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_int)]),
    "fd_autotune_fwi": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(fd_tile_config),
                                       ctypes.POINTER(fd_tile_config), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]),
    "fd_kernel_launches": (_i64, [_vp]),
    "fd_field_elems": (_i64, [_vp]),
    "fd_snapshot": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_restore": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_imaging": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_double]),
    "fd_step_fwi": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double]),
    "fd_run_fwi": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _i64, ctypes.c_int, _vp,
                                  ctypes.c_double]),
    "fd_residual": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "fd_field_to_dense": (ctypes.c_int, [_vp, _vp, _vp]),
    "fd_destroy": (None, [_vp]),
    "fd_last_error": (ctypes.c_char_p, [_vp]),
    "fd_weights": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "fd_stability_symbol": (ctypes.c_double, [ctypes.c_int]),
    "fd_version": (ctypes.c_char_p, []),
    "fd_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_double)]),
    "fd_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "fd_batch_add": (ctypes.c_int, [_vp, _vp]),
    "fd_batch_remove": (ctypes.c_int, [_vp, _vp]),
    "fd_batch_run": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_batch_size": (ctypes.c_int, [_vp]),
    "fd_batch_kernel_launches": (_i64, [_vp]),
    "fd_batch_last_error": (ctypes.c_char_p, [_vp]),
    "fd_batch_destroy": (None, [_vp]),
    "fd_footprint_bytes": (_i64, [ctypes.c_int, ctypes.POINTER(_i64), ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int]),
    "fd_acoustic_run_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_i64),
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                               ctypes.c_double, _vp, _vp, _vp, _vp, ctypes.c_int,
                                               _vp, _vp, _vp]),
}


def load(path=None):
    """Load libfd_b300.so (raises OSError if it is missing or unloadable)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError(f"CUDA library {p} is missing: build it with paper_1906_10811_b300.build.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(ctx, st):
    if st != FD_OK:
        msg = load().fd_last_error(ctx)
        raise FdError(st, msg.decode() if msg else "")


def _ptr(x, keep):
    """Address of a float32 C-contiguous array (numpy host array or torch tensor, or an
    int taken as a raw address).  A torch tensor of another dtype or layout is
    converted on torch's current stream: a caller whose library work runs on another
    stream must order that stream after the conversion (``Solver`` converts before
    it orders its stream)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):                       # torch tensor
        import torch
        t = x.detach()
        if t.dtype != torch.float32 or not t.is_contiguous():
            t = t.to(torch.float32).contiguous()
        keep.append(t)
        return t.data_ptr()
    a = np.ascontiguousarray(x, dtype=np.float32)
    keep.append(a)
    return a.ctypes.data


def _out_ptr(x):
    """Address of a preallocated float32 C-contiguous output (no conversion)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        import torch
        assert x.dtype == torch.float32 and x.is_contiguous(), "outputs must be float32 contiguous"
        return x.data_ptr()
    assert x.dtype == np.float32 and x.flags.c_contiguous, "outputs must be float32 C-contiguous"
    return x.ctypes.data


def options(nu=0.5, cuda_stream=None, device_ptrs=False, use_graphs=True, profile=False,
            kernel=FD_KERNEL_AUTO, autotune=False, boundary=FD_BOUNDARY_ZERO,
            dirichlet_interior=True):
    o = fd_options()
    load().fd_options_default(ctypes.byref(o))
    o.nu = nu
    o.cuda_stream = cuda_stream
    o.device_ptrs = int(bool(device_ptrs))
    o.use_graphs = int(bool(use_graphs))
    o.profile = int(bool(profile))
    o.kernel = int(kernel)
    o.autotune = int(bool(autotune))
    o.boundary = int(boundary)
    o.dirichlet_interior = int(bool(dirichlet_interior))
    return o


def fd_options_default():
    o = fd_options()
    load().fd_options_default(ctypes.byref(o))
    return o


def fd_create(ndim, shape, spacing, space_order, dt, eq, opt=None):
    lib = load()
    shp = (_i64 * max(ndim, 1))(*[int(s) for s in shape][:max(ndim, 1)])
    sp = (ctypes.c_double * max(ndim, 1))(*[float(h) for h in spacing][:max(ndim, 1)])
    out = _vp()
    st = lib.fd_create(ctypes.byref(out), ndim, shp, sp, int(space_order), float(dt), int(eq),
                       ctypes.byref(opt) if opt is not None else None)
    if st != FD_OK:
        raise FdError(st, lib.fd_last_error(None).decode())
    return out.value


def fd_set_model(ctx, m, damp=None):
    keep = []
    _check(ctx, load().fd_set_model(ctx, _ptr(m, keep), _ptr(damp, keep)))


def fd_set_field(ctx, u_cur, u_prev=None):
    keep = []
    _check(ctx, load().fd_set_field(ctx, _ptr(u_cur, keep), _ptr(u_prev, keep)))


def fd_set_sources(ctx, nsrc, coords, nt, wavelets):
    keep = []
    _check(ctx, load().fd_set_sources(ctx, int(nsrc), _ptr(coords, keep), int(nt),
                                      _ptr(wavelets, keep)))


def fd_set_receivers(ctx, nrec, coords):
    keep = []
    _check(ctx, load().fd_set_receivers(ctx, int(nrec), _ptr(coords, keep)))


def fd_run(ctx, nt):
    _check(ctx, load().fd_run(ctx, int(nt)))


def fd_read(ctx, u=None, rec=None):
    """Fill the given preallocated outputs (numpy float32 or torch float32)."""
    _check(ctx, load().fd_read(ctx, _out_ptr(u), _out_ptr(rec)))


def fd_read_prev(ctx, u_prev):
    _check(ctx, load().fd_read_prev(ctx, _out_ptr(u_prev)))


def fd_set_step(ctx, n):
    _check(ctx, load().fd_set_step(ctx, int(n)))


def fd_reset(ctx):
    _check(ctx, load().fd_reset(ctx))


def fd_steps_done(ctx):
    return int(load().fd_steps_done(ctx))


def fd_profile(ctx):
    """(launches, stencil_ms) since the previous call."""
    n = _i64()
    ms = ctypes.c_double()
    _check(ctx, load().fd_profile(ctx, ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def fd_kernel_name(ctx):
    return load().fd_kernel_name(ctx).decode()


def fd_skip_c_planes(ctx):
    """(flagged, total): tile-planes whose C tile the pipelined kernel skips."""
    f, t = _i64(), _i64()
    _check(ctx, load().fd_skip_c_planes(ctx, ctypes.byref(f), ctypes.byref(t)))
    return int(f.value), int(t.value)


def fd_set_subdomain(ctx, z_origin, z_global):
    _check(ctx, load().fd_set_subdomain(ctx, int(z_origin), int(z_global)))


def fd_halo_elems(ctx):
    return int(load().fd_halo_elems(ctx))


def fd_halo_copy(dst, side, src):
    _check(dst, load().fd_halo_copy(dst, int(side), src))


def fd_halo_export(ctx, side, dst):
    _check(ctx, load().fd_halo_export(ctx, int(side), _out_ptr(dst)))


def fd_halo_import(ctx, side, src):
    _check(ctx, load().fd_halo_import(ctx, int(side), _ptr(src, [])))


def fd_run_slabs(ctxs, nt):
    arr = (_vp * len(ctxs))(*ctxs)
    st = load().fd_run_slabs(arr, len(ctxs), int(nt))
    if st != FD_OK:
        bad = [c for c in ctxs if load().fd_last_error(c)]
        msg = load().fd_last_error(bad[-1] if bad else None)
        raise FdError(st, msg.decode() if msg else "")


def fd_accumulate_traces(ctx, acc):
    _check(ctx, load().fd_accumulate_traces(ctx, _out_ptr(acc)))


def fd_get_tile_config(ctx):
    """The pipelined kernel's tile configuration as a dict."""
    cfg = fd_tile_config()
    st = load().fd_get_tile_config(ctx, ctypes.byref(cfg))
    if st != FD_OK:
        raise FdError(st, "no tile configuration (plain kernel)")
    return cfg.as_dict()


def fd_set_tile_config(ctx, tile_y=0, zblock=0, ctas_per_sm=0, tile_x=0, aligned=0, skip_c=0):
    cfg = fd_tile_config(int(tile_x), int(tile_y), int(zblock), int(ctas_per_sm), int(aligned),
                         int(skip_c), 0.0)
    _check(ctx, load().fd_set_tile_config(ctx, ctypes.byref(cfg)))


def fd_autotune(ctx, reps=5, max_tried=256, fwi=False):
    """Time the tile configurations and use the fastest: (best, tried) as dicts.

    fwi: time them as the FWI sweep's kernels (fd_autotune_fwi).  max_tried = 0
    passes no list, so an earlier choice for the same problem is reused."""
    best = fd_tile_config()
    tried = (fd_tile_config * max_tried)() if max_tried > 0 else None
    n = ctypes.c_int()
    fn = load().fd_autotune_fwi if fwi else load().fd_autotune
    _check(ctx, fn(ctx, int(reps), ctypes.byref(best), tried, int(max_tried), ctypes.byref(n)))
    return best.as_dict(), ([tried[i].as_dict() for i in range(min(n.value, max_tried))]
                            if tried else [])


def fd_kernel_launches(ctx):
    return int(load().fd_kernel_launches(ctx))


def _bcheck(batch, st):
    if st != FD_OK:
        msg = load().fd_batch_last_error(batch) if batch else load().fd_last_error(None)
        raise FdError(st, msg.decode() if msg else "")


def fd_batch_create(space_order, cuda_stream=None):
    out = _vp()
    st = load().fd_batch_create(ctypes.byref(out), int(space_order), cuda_stream)
    _bcheck(None, st)
    return out.value


def fd_batch_add(batch, ctx):
    _bcheck(batch, load().fd_batch_add(batch, ctx))


def fd_batch_remove(batch, ctx):
    _bcheck(batch, load().fd_batch_remove(batch, ctx))


def fd_batch_run(batch, nticks):
    _bcheck(batch, load().fd_batch_run(batch, int(nticks)))


def fd_batch_size(batch):
    return int(load().fd_batch_size(batch))


def fd_batch_kernel_launches(batch):
    return int(load().fd_batch_kernel_launches(batch))


def fd_batch_destroy(batch):
    if batch:
        load().fd_batch_destroy(batch)


def fd_footprint_bytes(shape, space_order, nrec, nt, nsrc=1):
    nd = len(shape)
    shp = (_i64 * nd)(*[int(x) for x in shape])
    return int(load().fd_footprint_bytes(nd, shp, int(space_order), int(nrec), int(nt), int(nsrc)))


def fd_field_elems(ctx):
    return int(load().fd_field_elems(ctx))


def fd_snapshot(ctx, dst_cur, dst_prev=None):
    _check(ctx, load().fd_snapshot(ctx, _out_ptr(dst_cur), _out_ptr(dst_prev)))


def fd_restore(ctx, src_cur, src_prev):
    _check(ctx, load().fd_restore(ctx, _ptr(src_cur, []), _ptr(src_prev, [])))


def fd_imaging(adj, g, u_next, u_cur, u_prev, scale):
    _check(adj, load().fd_imaging(adj, _out_ptr(g), _ptr(u_next, []), _ptr(u_cur, []),
                                  _ptr(u_prev, []), float(scale)))


def fd_step_fwi(ctx, d2_out=None, img_g=None, img_d2=None, scale=0.0):
    keep = []
    _check(ctx, load().fd_step_fwi(ctx, _out_ptr(d2_out), _out_ptr(img_g), _ptr(img_d2, keep),
                                   float(scale)))


def fd_run_fwi(ctx, nt, d2_base=None, img_d2_base=None, stride=0, reverse=False, img_g=None,
               scale=0.0):
    """nt FWI-epilogue steps; step i uses row s of the [nt][stride] bases, s = i or nt-1-i."""
    _check(ctx, load().fd_run_fwi(ctx, int(nt), _out_ptr(d2_base), _ptr(img_d2_base, []),
                                  int(stride), int(bool(reverse)), _out_ptr(img_g), float(scale)))


def fd_residual(ctx, d_obs, adj_wav=None):
    """J = ½||traces − d_obs||² (float); adj_wav (if given) receives the residual time
    reversed, the adjoint run's source wavelet."""
    J = ctypes.c_double()
    _check(ctx, load().fd_residual(ctx, _ptr(d_obs, []), _out_ptr(adj_wav), ctypes.byref(J)))
    return float(J.value)


def fd_field_to_dense(ctx, padded, dense):
    _check(ctx, load().fd_field_to_dense(ctx, _ptr(padded, []), _out_ptr(dense)))


def fd_destroy(ctx):
    if ctx:
        load().fd_destroy(ctx)


def fd_last_error(ctx=None):
    return load().fd_last_error(ctx).decode()


def fd_weights(space_order):
    w = (ctypes.c_double * 9)()
    st = load().fd_weights(int(space_order), w)
    if st != FD_OK:
        raise FdError(st, f"bad space order {space_order}")
    return [w[k] for k in range(space_order // 2 + 1)]


def fd_stability_symbol(space_order):
    return float(load().fd_stability_symbol(int(space_order)))


def fd_selftest_bounded_wait(budget_ms):
    """(expired, waited_ms) of a bounded wait on a barrier nothing completes."""
    ex = ctypes.c_int()
    ms = ctypes.c_double()
    st = load().fd_selftest_bounded_wait(float(budget_ms), ctypes.byref(ex), ctypes.byref(ms))
    if st != FD_OK:
        raise FdError(st, load().fd_last_error(None).decode())
    return bool(ex.value), float(ms.value)


def fd_version():
    return load().fd_version().decode()


def fd_acoustic_run_noalloc(shape, spacing, space_order, dt, m, damp, u_cur, u_prev, nt, u_out,
                            u_prev_out=None, cuda_stream=None):
    """No-allocation acoustic run on caller-owned device tensors (see include/fd.h).

    For callers that cannot allocate GPU memory.  Every array argument is a
    float32, C-contiguous torch CUDA tensor on the current device holding
    prod(shape) elements (damp, u_prev and u_prev_out may be None); anything
    else raises before the library is called, since the library receives bare
    pointers and cannot check sizes itself.  Nothing is converted or copied
    here.  cuda_stream: a torch stream or a cudaStream_t handle; default the
    current torch stream, so that work queued there before the call (the
    tensors' producers) is ordered before it.
    """
    import torch
    n = int(np.prod([int(x) for x in shape])) if len(shape) else 0
    dev = torch.cuda.current_device()
    args = dict(m=m, damp=damp, u_cur=u_cur, u_prev=u_prev, u_out=u_out, u_prev_out=u_prev_out)
    for name, x in args.items():
        if x is None:
            if name in ("m", "u_cur", "u_out"):
                raise ValueError(f"{name} is required")
            continue
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError(f"{name}: fd_acoustic_run_noalloc takes torch CUDA tensors only")
        if x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError(f"{name}: must be float32 and contiguous (no conversion is made)")
        if x.device.index != dev:
            raise ValueError(f"{name} is on cuda:{x.device.index}, the current device is cuda:{dev}")
        if x.numel() != n:
            raise ValueError(f"{name} holds {x.numel()} elements, the grid has {n}")
    if cuda_stream is None:
        cuda_stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(cuda_stream, "cuda_stream"):
        cuda_stream = cuda_stream.cuda_stream
    lib = load()
    nd = len(shape)
    shp = (_i64 * nd)(*[int(x) for x in shape])
    sp = (ctypes.c_double * nd)(*[float(h) for h in spacing])
    ptr = lambda x: None if x is None else x.data_ptr()
    st = lib.fd_acoustic_run_noalloc(nd, shp, sp, int(space_order), float(dt), ptr(m), ptr(damp),
                                     ptr(u_cur), ptr(u_prev), int(nt), ptr(u_out),
                                     ptr(u_prev_out), cuda_stream)
    if st != FD_OK:
        raise FdError(st, lib.fd_last_error(None).decode())
