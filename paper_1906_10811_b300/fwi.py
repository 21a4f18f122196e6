"""Full-waveform-inversion gradient on the device (adjoint state, checkpointing).

J(m) = ½ Σ_n ||P_r u^n(m) − d_obs^n||² for one acoustic shot.  The gradient
comes from the exact adjoint of the discrete leapfrog: with ν = a·λ
(a = dt²/(m+σ)) the adjoint recursion is the forward scheme run backwards,

    ν^k = a·L ν^{k+1} + b·ν^{k+1} − c·ν^{k+2} + a·P_rᵀ r^k,     k = N .. 1,

so the adjoint is the library's own solver with the receivers acting as
sources (wavelet = the residual, time reversed; where damp = 0 the injection
w·dt²/m equals a·w), and

    dJ/dm = −(1/dt²) Σ_n ν^{n+1} ⊙ (u^{n+1} − 2u^n + u^{n−1}),

accumulated by the library's imaging-condition kernel (fd_imaging, or the
stencil epilogue through fd_step_fwi / fd_run_fwi).  The residual, the misfit J
and the time-reversed adjoint wavelet come from fd_residual.  The
forward wavefield is needed backwards in time: it is checkpointed every k
steps (fd_snapshot) and each block of k steps is recomputed from its
checkpoint while the adjoint sweeps it; on the pipelined kernel the forward
sweep writes the last block's second differences itself, so that block is not
recomputed (and with k = nt nothing is).  ``choose_checkpoint_interval`` picks
the largest k the device memory allows; ``tune_checkpoint_interval`` times
the candidates and keeps the fastest (the least memory among near-ties).  Every
arithmetic step runs in CUDA kernels; this module orders them (torch holds the
device memory and the stream).
"""

import math

import numpy as np

from . import binding as B
from .solver import Solver


def _dev():
    import torch
    return torch


def choose_checkpoint_interval(nt, field_bytes, budget_bytes):
    """Largest k whose memory fits: (k + 2) block levels + 2·ceil(nt/k) checkpoint levels.

    k = nt keeps every level (no recompute beyond one pass)."""
    best = 1
    for k in range(1, nt + 1):
        need = (k + 2 + 2 * math.ceil(nt / k)) * field_bytes
        if need <= budget_bytes:
            best = k
    return best


def blocks(nt, k):
    """Checkpoint blocks [(n0, n1)] of at most k steps: the short one first, so that
    the last block, whose second differences the forward sweep writes itself (no
    recompute), is a full k steps."""
    nblk = math.ceil(nt / k)
    starts = [max(0, nt - (nblk - c) * k) for c in range(nblk)]
    return list(zip(starts, starts[1:] + [nt]))


def checkpoint_memory(nt, k, field_bytes):
    """Device bytes of checkpoint-every-k: 2·ceil(nt/k) checkpoint levels + k+2 block levels."""
    return (k + 2 + 2 * math.ceil(nt / k)) * field_bytes


def checkpoint_candidates(nt, field_bytes, budget_bytes):
    """Intervals worth timing: the least-memory k (about √(2 nt)), a few multiples of
    it, nt/4, nt/2 and the largest k that fits the budget."""
    kmax = choose_checkpoint_interval(nt, field_bytes, budget_bytes)
    kmin = min(range(1, nt + 1), key=lambda k: (checkpoint_memory(nt, k, field_bytes), k))
    cands = {kmin, 2 * kmin, 4 * kmin, nt // 4, nt // 2, kmax}
    return sorted(c for c in cands if 1 <= c <= kmax)


def tune_checkpoint_interval(p, d_obs, m=None, candidates=None, memory_budget=None, tol=0.03):
    """Pick the checkpoint interval by timing one gradient per candidate.

    Every block but the last is recomputed (nt minus the last block's steps),
    so larger k recompute less but hold more memory; the fastest k wins, except
    that a candidate within ``tol`` of it that holds less memory is preferred.
    Each candidate's time includes mapping its buffers (one gradient from a
    clean allocator): at 320³ × 1000 steps the candidates above ~80 GB were
    slower even on repeated gradients.  Returns (k, [(k, seconds, bytes)]).
    """
    torch = _dev()
    nt = p["nt"]
    with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", device=True) as s:
        field_bytes = B.fd_field_elems(s.ctx) * 4
    if memory_budget is None:
        free, _ = torch.cuda.mem_get_info()
        memory_budget = int(0.6 * free)
    if candidates is None:
        candidates = checkpoint_candidates(nt, field_bytes, memory_budget)
    gradient(p, d_obs, m=m, k=candidates[0])   # untimed: first-use costs (graphs, pools)
    torch.cuda.empty_cache()
    rows = []
    for k in candidates:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gradient(p, d_obs, m=m, k=k)
        e1.record()
        e1.synchronize()
        rows.append((int(k), e0.elapsed_time(e1) / 1e3, checkpoint_memory(nt, k, field_bytes)))
        torch.cuda.empty_cache()          # the next candidate's buffers differ in size
    fastest = min(r[1] for r in rows)
    ok = [r for r in rows if r[1] <= fastest * (1.0 + tol)]
    best = min(ok, key=lambda r: (r[2], r[1]))
    return best[0], rows


def _check_sparse_undamped(p):
    """The adjoint identities used here need damp = 0 at every sparse corner node."""
    damp = np.asarray(p["damp"]) if p.get("damp") is not None else None
    if damp is None:
        return
    shape, h = p["shape"], p["spacing"]
    for c in list(p["src_coords"]) + list(p["rec_coords"]):
        idx, frac = [], []
        for d, (n, hd) in enumerate(zip(shape, h)):
            x = min(max(float(c[d]) / hd, 0.0), n - 1.0)
            i = min(int(math.floor(x)), n - 2)
            idx.append((i, i + 1))
            frac.append((1.0 - (x - i), x - i))
        for corner in np.ndindex(*(2,) * len(shape)):
            if any(frac[d][corner[d]] == 0.0 for d in range(len(shape))):
                continue                                   # zero-weight corner
            node = tuple(idx[d][corner[d]] for d in range(len(shape)))
            if damp[node] != 0.0:
                raise ValueError("sources and receivers must lie where damp = 0")


def forward_traces(p, m=None):
    """Traces [nt+1][nrec] (torch, device) of shot p with model m (torch or numpy)."""
    torch = _dev()
    mm = p["m"] if m is None else m
    with Solver(p["shape"], p["spacing"], p["so"], p["dt"], "acoustic", device=True) as s:
        s.set_model(torch.as_tensor(mm, dtype=torch.float32, device="cuda"),
                    torch.as_tensor(p["damp"], dtype=torch.float32, device="cuda"))
        s.set_sources(torch.as_tensor(p["src_coords"], device="cuda"),
                      torch.as_tensor(p["wavelet"], device="cuda"))
        s.set_receivers(torch.as_tensor(p["rec_coords"], device="cuda"))
        s.run(p["nt"])
        _, rec = s.read(field=False)
    return rec


def gradient(p, d_obs, m=None, k=None, memory_budget=None, stats=None, profile=False,
             fused=None):
    """(J, dJ/dm) for shot p (fdsynth.acoustic_problem layout) against d_obs.

    m: model (defaults to p["m"]); k: checkpoint interval (None: chosen from
    the free device memory or ``memory_budget`` bytes).  Returns a float and a
    torch tensor shaped like m on the device.  ``stats`` (a dict, optional)
    receives k, the device bytes held for checkpoints and the recompute block,
    and the kernel launches of the forward and adjoint contexts; with
    ``profile`` also their stencil launches and summed stencil milliseconds
    (CUDA events around each replayed chunk of steps).  ``fused`` (default:
    wherever the pipelined 3-D kernel runs) takes the backward sweep through
    fd_run_fwi, the second time difference and the imaging condition computed
    in the stencil epilogues and the steps of a block replayed from CUDA graphs;
    the result is bitwise the same.
    """
    torch = _dev()
    _check_sparse_undamped(p)
    caller = torch.cuda.current_stream()
    work = torch.cuda.Stream()            # both contexts and every copy on one stream
    work.wait_stream(caller)
    with torch.cuda.stream(work):
        J, g = _gradient_on_stream(p, d_obs, m, k, memory_budget, stats, profile, fused)
    caller.wait_stream(work)
    return J, g


def _gradient_on_stream(p, d_obs, m, k, memory_budget, stats=None, profile=False, fused=None):
    torch = _dev()
    nt, dt = p["nt"], p["dt"]
    mm = torch.as_tensor(p["m"] if m is None else m, dtype=torch.float32, device="cuda")
    damp = torch.as_tensor(p["damp"], dtype=torch.float32, device="cuda")
    src = torch.as_tensor(p["src_coords"], device="cuda")
    wav = torch.as_tensor(p["wavelet"], device="cuda")
    rc = torch.as_tensor(p["rec_coords"], device="cuda")
    d_obs = torch.as_tensor(d_obs, dtype=torch.float32, device="cuda")

    fwd = Solver(p["shape"], p["spacing"], p["so"], dt, "acoustic", device=True, profile=profile)
    adj = Solver(p["shape"], p["spacing"], p["so"], dt, "acoustic", device=True, profile=profile)
    try:
        fwd.set_model(mm, damp)
        if fwd.kernel_name in ("stencil3d_tma_acoustic", "stencil3d_xp_acoustic"):
            # both contexts take the tile timed on the sweep's own kernels (cached per grid)
            fwd.autotune(fwi=True, cached=True)
            t = fwd.tile_config
            adj.set_tile_config(tile_y=t["tile_y"], zblock=t["zblock"],
                                ctas_per_sm=t["ctas_per_sm"], aligned=t["aligned"],
                                skip_c=t["skip_c"])
        fwd.set_sources(src, wav)
        fwd.set_receivers(rc)
        elems = B.fd_field_elems(fwd.ctx)
        if k is None:
            if memory_budget is None:
                free, _ = torch.cuda.mem_get_info()
                memory_budget = int(0.6 * free)
            k = choose_checkpoint_interval(nt, elems * 4, memory_budget)
        k = max(1, min(int(k), nt))
        blk_range = blocks(nt, k)
        nblk = len(blk_range)
        if fused is None:
            fused = len(p["shape"]) == 3 and fwd.kernel_name == "stencil3d_tma_acoustic"
        ck = torch.empty((nblk, 2, elems), dtype=torch.float32, device="cuda")
        # fused: the second differences of one block, u^{n+1} − 2u^n + u^{n−1}
        blk = torch.empty((k, elems), dtype=torch.float32, device="cuda") if fused else None
        # forward sweep with checkpoints (u^{ck}, u^{ck-1}) at the start of each block;
        # fused, the last block's steps also write its second differences
        for c, (n0, n1) in enumerate(blk_range):
            B.fd_snapshot(fwd.ctx, ck[c, 0], ck[c, 1])
            if fused and c == nblk - 1:      # step t writes its second difference to blk[t - n0]
                B.fd_run_fwi(fwd.ctx, n1 - n0, d2_base=blk, stride=elems)
            else:
                fwd.run(n1 - n0)
        # residual r = traces − d_obs, J = ½||r||² and the adjoint source wavelet
        # (row j = r[nt − j]) in the library
        adj_wav = torch.empty((nt, rc.shape[0]), dtype=torch.float32, device="cuda")
        J = B.fd_residual(fwd.ctx, d_obs, adj_wav)
        # adjoint: sources at the receivers
        adj.set_model(mm, damp)
        adj.set_sources(rc, adj_wav)
        B.fd_set_receivers(fwd.ctx, 0, None)
        scale = -1.0 / (dt * dt)
        if fused:
            # the recompute writes u^{n+1} − 2u^n + u^{n−1} from its own epilogue and
            # the adjoint step accumulates the imaging condition from its epilogue
            g = torch.empty(p["shape"], dtype=torch.float32, device="cuda")
            gp = torch.zeros(elems, dtype=torch.float32, device="cuda")
            for c in range(nblk - 1, -1, -1):
                n0, n1 = blk_range[c]
                if c < nblk - 1:   # the last block's differences are in blk already
                    B.fd_restore(fwd.ctx, ck[c, 0], ck[c, 1])
                    fwd.set_step(n0)
                    B.fd_run_fwi(fwd.ctx, n1 - n0, d2_base=blk, stride=elems)
                # adjoint step nt-1-n gives ν^{n+1} and reads blk[n - n0]: the block backwards
                B.fd_run_fwi(adj.ctx, n1 - n0, img_d2_base=blk, stride=elems, reverse=True,
                             img_g=gp, scale=scale)
            B.fd_field_to_dense(fwd.ctx, gp, g)
            blk_bytes = int(blk.numel() + gp.numel()) * 4
        else:
            g, blk_bytes = _backward_unfused(p, fwd, adj, ck, k, blk_range, elems, scale)
        if stats is not None:
            stats.update(k=k, checkpoint_bytes=int(ck.numel()) * 4, block_bytes=blk_bytes,
                         fused=bool(fused),
                         tile=fwd.tile_config if fwd.kernel_name.startswith("stencil3d_tma")
                         else None,
                         launches_forward=fwd.kernel_launches, launches_adjoint=adj.kernel_launches)
            if profile:
                nf, msf = fwd.profile()
                na, msa = adj.profile()
                stats.update(stencil_launches=nf + na, stencil_ms=msf + msa)
        torch.cuda.current_stream().synchronize()
        return J, g
    finally:
        fwd.close()
        adj.close()


def _backward_unfused(p, fwd, adj, ck, k, blk_range, elems, scale):
    """Backward sweep with separate kernels: recompute + snapshot, adjoint step, imaging."""
    torch = _dev()
    g = torch.zeros(p["shape"], dtype=torch.float32, device="cuda")
    blk = torch.empty((k + 2, elems), dtype=torch.float32, device="cuda")
    for c in range(len(blk_range) - 1, -1, -1):
        n0, n1 = blk_range[c]
        # recompute u^{n0-1} .. u^{n1} into blk[0 .. n1-n0+1]
        B.fd_restore(fwd.ctx, ck[c, 0], ck[c, 1])
        fwd.set_step(n0)
        blk[0].copy_(ck[c, 1])
        blk[1].copy_(ck[c, 0])
        for t in range(n0, n1):
            fwd.run(1)
            B.fd_snapshot(fwd.ctx, blk[t - n0 + 2])
        for n in range(n1 - 1, n0 - 1, -1):       # adjoint step nt-1-n gives ν^{n+1}
            adj.run(1)
            i = n - n0 + 1                          # blk[i] = u^n
            B.fd_imaging(adj.ctx, g, blk[i + 1], blk[i], blk[i - 1], scale)
    return g, int(blk.numel()) * 4


class FWIObjective:
    """``torch.autograd.Function`` wrapper: J = FWIObjective.apply(m, p, d_obs, k).

    The forward pass computes J and, with it, dJ/dm (the adjoint sweep reuses
    the checkpoints of the same forward run); backward scales the stored
    gradient by the incoming gradient.
    """

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            torch = _dev()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, m, p, d_obs, k):
                    J, g = gradient(p, d_obs, m=m.detach(), k=k)
                    ctx.save_for_backward(g)
                    return torch.tensor(J, dtype=torch.float64, device=m.device)

                @staticmethod
                def backward(ctx, grad_out):
                    (g,) = ctx.saved_tensors
                    return (grad_out.to(g.dtype) * g), None, None, None

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, m, p, d_obs, k=None):
        return cls.function().apply(m, p, d_obs, k)
