"""``Solver``: a Python object over one fd_ctx (marshalling only; all work runs in
the CUDA library).  Host mode takes and returns numpy arrays; device mode
(``device=True``) takes and returns torch CUDA tensors.  Device mode runs on the
caller's current torch stream, or, when that is the legacy default stream
(which cannot be captured into graphs), on a private stream that is ordered
after the caller's stream before every call and before the caller's stream
after every call."""

import numpy as np

from . import binding as B

_EQ = {"diffusion": B.FD_DIFFUSION, "acoustic": B.FD_ACOUSTIC}
_KERNEL = {"auto": B.FD_KERNEL_AUTO, "plain": B.FD_KERNEL_PLAIN, "tma": B.FD_KERNEL_TMA}
_BOUNDARY = {"zero": B.FD_BOUNDARY_ZERO, "odd": B.FD_BOUNDARY_ODD}


class Solver:
    """One simulation: ``Solver(shape, spacing, space_order, dt, equation)``.

    Mirrors a Devito operator's problem statement (thesis §2.1.1: a Grid with
    shape and spacing, a TimeFunction of a space order, initial data, sparse
    sources/receivers, ``op(time=nt, dt=dt)``).
    """

    def __init__(self, shape, spacing, space_order, dt, equation="acoustic", nu=0.5,
                 device=False, stream=None, graphs=True, profile=False, kernel="auto",
                 autotune=False, boundary="zero", dirichlet_interior=True):
        self.ctx = None
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.device = bool(device)
        cuda_stream = None
        self._private = False
        if self.device:
            import torch
            self._torch = torch
            s = stream if stream is not None else torch.cuda.current_stream()
            if s.cuda_stream == 0:
                # the legacy default stream cannot host graph capture: work on a
                # private stream, ordered with the caller's stream at every call
                s = torch.cuda.Stream()
                self._private = True
            cuda_stream = s.cuda_stream
            self.stream = s
        opt = B.options(nu=nu, cuda_stream=cuda_stream, device_ptrs=self.device, use_graphs=graphs,
                        profile=profile, kernel=_KERNEL[kernel], autotune=autotune,
                        boundary=_BOUNDARY[boundary], dirichlet_interior=dirichlet_interior)
        self._in()
        self.ctx = B.fd_create(self.ndim, self.shape, spacing, space_order, dt, _EQ[equation], opt)
        self._out()
        self.nrec = 0

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            B.fd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stream ordering (device mode on a private stream) ------------------
    def _in(self):
        """The solver's stream waits for work already queued by the caller."""
        if self._private:
            self.stream.wait_stream(self._torch.cuda.current_stream())

    def _out(self):
        """The caller's stream waits for the solver's work."""
        if self._private:
            self._torch.cuda.current_stream().wait_stream(self.stream)

    # -- inputs ------------------------------------------------------------
    def _f32(self, x):
        """Device mode: a float32 contiguous tensor, converted on the caller's stream
        before the solver's stream is ordered after it (so the library reads the
        converted copy, not memory still being written)."""
        if x is None or not self.device or not hasattr(x, "data_ptr"):
            return x
        torch = self._torch
        if x.dtype != torch.float32 or not x.is_contiguous():
            x = x.to(torch.float32).contiguous()
        return x

    def set_model(self, m, damp=None):
        m, damp = self._f32(m), self._f32(damp)
        self._in()
        B.fd_set_model(self.ctx, m, damp)

    def set_field(self, u, u_prev=None):
        u, u_prev = self._f32(u), self._f32(u_prev)
        self._in()
        B.fd_set_field(self.ctx, u, u_prev)
        self._out()

    def set_sources(self, coords, wavelets):
        coords, wavelets = self._f32(coords), self._f32(wavelets)
        self._in()
        n = 0 if coords is None else len(coords)
        nt = 0 if wavelets is None else int(wavelets.shape[0])
        B.fd_set_sources(self.ctx, n, coords, nt, wavelets)

    def set_receivers(self, coords):
        coords = self._f32(coords)
        self._in()
        self.nrec = 0 if coords is None else len(coords)
        B.fd_set_receivers(self.ctx, self.nrec, coords)

    def set_step(self, n):
        B.fd_set_step(self.ctx, n)

    def reset(self):
        """Back to rest: both levels zero, step 0, traces cleared (no upload)."""
        self._in()
        B.fd_reset(self.ctx)
        self._out()

    # -- run / outputs -----------------------------------------------------
    def run(self, nt):
        self._in()
        B.fd_run(self.ctx, nt)
        self._out()
        return self

    @property
    def steps(self):
        return B.fd_steps_done(self.ctx)

    @property
    def kernel_name(self):
        return B.fd_kernel_name(self.ctx)

    @property
    def kernel_launches(self):
        return B.fd_kernel_launches(self.ctx)

    def skipped_c_planes(self):
        """(flagged, total): tile-planes whose C tile the pipelined kernel skips."""
        self._in()
        out = B.fd_skip_c_planes(self.ctx)
        self._out()
        return out

    # -- tile configuration of the pipelined 3-D kernel ----------------------
    @property
    def tile_config(self):
        """{tile_x, tile_y, zblock, ctas_per_sm, aligned, skip_c, us_per_step} of the pipelined kernel."""
        return B.fd_get_tile_config(self.ctx)

    def set_tile_config(self, tile_y=0, zblock=0, ctas_per_sm=0, aligned=0, skip_c=0, tile_x=0):
        """Tile configuration of the pipelined 3-D kernel (fd_set_tile_config): tile_x 32
        or 64 (two x points a lane), tile_y 16 or 32 (24 with tile_x 64 from space order
        8: 12 consumer warps), split aligned 0 (equal ranges), 1 (whole segments) or 2
        (work queue, tile_x 64), skip_c 1 to skip C where it is 1; 0 means the default.
        Every configuration computes the same bits."""
        self._in()
        B.fd_set_tile_config(self.ctx, tile_y=tile_y, zblock=zblock, ctas_per_sm=ctas_per_sm,
                             aligned=aligned, skip_c=skip_c, tile_x=tile_x)
        self._out()

    def autotune(self, reps=5, fwi=False, cached=False):
        """Time every tile configuration and keep the fastest: (best, tried).

        fwi: time them as one backward step of the FWI sweep (fd_autotune_fwi);
        cached: reuse the process's earlier choice for this problem if there is
        one (``tried`` is then empty)."""
        self._in()
        out = B.fd_autotune(self.ctx, reps=reps, fwi=fwi, max_tried=0 if cached else 256)
        self._out()
        return out

    def _empty(self, shape):
        if self.device:
            return self._torch.empty(shape, dtype=self._torch.float32, device="cuda")
        return np.empty(shape, dtype=np.float32)

    def read(self, field=True, traces=True):
        """(u^n, traces [n+1][nrec]); either is None when not requested or absent."""
        self._in()
        u = self._empty(self.shape) if field else None
        rec = self._empty((self.steps + 1, self.nrec)) if traces and self.nrec else None
        B.fd_read(self.ctx, u, rec)
        self._out()
        return u, rec

    def read_prev(self):
        self._in()
        u = self._empty(self.shape)
        B.fd_read_prev(self.ctx, u)
        self._out()
        return u

    def profile(self):
        """(stencil launches, summed stencil ms) since the previous call."""
        return B.fd_profile(self.ctx)


class Batch:
    """Shots of one space order stepped together (see fd_batch_* in include/fd.h).

    ``add``/``remove`` take :class:`Solver` objects; ``run(n)`` advances every
    member n steps with one set of batched launches per step.  A member keeps
    its own state, so ``Solver.read`` works on it afterwards.
    """

    def __init__(self, space_order, stream=None):
        self.handle = None
        cs = None
        if stream is not None:
            cs = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        self.handle = B.fd_batch_create(space_order, cs)
        self.members = []

    def add(self, solver):
        B.fd_batch_add(self.handle, solver.ctx)
        self.members.append(solver)

    def remove(self, solver):
        B.fd_batch_remove(self.handle, solver.ctx)
        self.members.remove(solver)

    def run(self, nticks):
        B.fd_batch_run(self.handle, nticks)

    @property
    def kernel_launches(self):
        return B.fd_batch_kernel_launches(self.handle)

    def __len__(self):
        return B.fd_batch_size(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.fd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
