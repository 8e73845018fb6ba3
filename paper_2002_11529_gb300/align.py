"""Detector alignment through the library's chi2 adjoint kernels.

The p-kick fit's chi2 (Sec. III-C) of tracks with fixed selected hits, as a
function of the track states theta [T,3] = (x, tx, qop) and the per-sector
alignment [4S,3] = (dx, dz, gamma), is exposed as a torch.autograd.Function
whose backward is the library's hand-written adjoint (ut_align_chi2).

solve_alignment estimates the alignment by preconditioned conjugate
gradients on the reduced Gauss-Newton system (track states profiled out by
a refit): every step is one reduced Hessian-vector product, the
preconditioner the per-sector 3x3 Gauss-Newton blocks; the whole loop runs
in the library (ut_align_solve), this module only marshals.  The detector
alone cannot fix three global modes (a layer-wise x shift proportional to
z - z_kink, absorbed by every track's q/p, and two z scalings about the kink
plane); starting from zero, the solver leaves them essentially untouched.
"""
from __future__ import annotations

import ctypes

import torch

from . import (_check, _ptr, _stream, lib, params_struct, HitBuffers, VeloBuffers)


class AlignmentProblem:
    """Tracks with fixed hits on the device, and the calls of the ABI."""

    def __init__(self, ctx, hits: HitBuffers, track_hits: torch.Tensor, velo: VeloBuffers, params):
        self.ctx = ctx
        self.hits = hits
        self.track_hits = track_hits.contiguous()
        self.velo = velo
        self.params = params
        self.n_tracks = int(track_hits.shape[0])
        self.S = int(ctx.geom.n_sectors)
        dev = track_hits.device
        nws = int(lib().ut_align_workspace_size(self.S))
        self.ws = torch.empty((nws + 7) // 8, dtype=torch.int64, device=dev)
        self._h = hits.struct()
        self._v = velo.struct()
        self._p = params_struct(params)

    def refit(self, align: torch.Tensor, stream=None) -> torch.Tensor:
        theta = torch.empty((self.n_tracks, 3), dtype=torch.float32, device=align.device)
        _check(lib().ut_align_refit(self.ctx.handle, ctypes.byref(self._h), ctypes.byref(self._v),
                                    _ptr(self.track_hits), self.n_tracks, ctypes.byref(self._p),
                                    _ptr(align.contiguous()), _ptr(theta), _stream(stream)), "ut_align_refit")
        return theta

    def chi2(self, theta: torch.Tensor, align: torch.Tensor, grads=False, stream=None):
        dev = align.device
        c2 = torch.empty(1, dtype=torch.float64, device=dev)
        gt = torch.empty((self.n_tracks, 3), dtype=torch.float32, device=dev) if grads else None
        ga = torch.empty((4 * self.S, 3), dtype=torch.float32, device=dev) if grads else None
        ha = torch.empty((4 * self.S, 6), dtype=torch.float32, device=dev) if grads else None
        _check(lib().ut_align_chi2(self.ctx.handle, ctypes.byref(self._h), ctypes.byref(self._v),
                                   _ptr(self.track_hits), self.n_tracks, ctypes.byref(self._p),
                                   _ptr(align.contiguous()), _ptr(theta.contiguous()), _ptr(c2), _ptr(gt),
                                   _ptr(ga), _ptr(ha), _ptr(self.ws), self.ws.numel() * 8, _stream(stream)),
               "ut_align_chi2")
        if not grads:
            return c2
        return c2, gt, ga, ha

    def hvp(self, theta: torch.Tensor, align: torch.Tensor, v: torch.Tensor, stream=None) -> torch.Tensor:
        hv = torch.empty((4 * self.S, 3), dtype=torch.float64, device=align.device)
        _check(lib().ut_align_hvp(self.ctx.handle, ctypes.byref(self._h), ctypes.byref(self._v),
                                  _ptr(self.track_hits), self.n_tracks, ctypes.byref(self._p),
                                  _ptr(align.contiguous()), _ptr(theta.contiguous()),
                                  _ptr(v.to(torch.float64).contiguous()), _ptr(hv), _stream(stream)),
               "ut_align_hvp")
        return hv


class Chi2Alignment(torch.autograd.Function):
    """chi2(theta, align) with the library's adjoint as backward."""

    @staticmethod
    def forward(ctx, theta, align, problem: AlignmentProblem):
        ctx.problem = problem
        ctx.save_for_backward(theta, align)
        return problem.chi2(theta.detach(), align.detach())[0]

    @staticmethod
    def backward(ctx, grad_out):
        theta, align = ctx.saved_tensors
        _, gt, ga, _ = ctx.problem.chi2(theta.detach(), align.detach(), grads=True)
        g = grad_out.to(torch.float32)
        return (g * gt if ctx.needs_input_grad[0] else None,
                g * ga if ctx.needs_input_grad[1] else None, None)


def solve_alignment(problem: AlignmentProblem, steps: int = 20, relinearize_every: int = 10,
                    align0: torch.Tensor | None = None, stream=None):
    """Estimate the alignment in `steps` preconditioned CG steps (one reduced
    Hessian-vector product each), re-linearising (refit, new gradient and
    blocks) every `relinearize_every` steps: one ut_align_solve call, the
    whole loop on the device.  Returns (align, history): the estimate [4S,3]
    and a device tensor of the chi2 at the start of each linearisation and
    at the estimate."""
    dev = problem.track_hits.device
    a = torch.zeros((4 * problem.S, 3), dtype=torch.float32, device=dev) if align0 is None else \
        align0.to(torch.float32).contiguous().clone()
    n_hist = (steps + relinearize_every - 1) // relinearize_every + 1
    history = torch.empty(n_hist, dtype=torch.float64, device=dev)
    nws = int(lib().ut_align_solve_workspace_size(problem.S, problem.n_tracks))
    ws = torch.empty((nws + 15) // 16 * 2, dtype=torch.float64, device=dev)
    _check(lib().ut_align_solve(problem.ctx.handle, ctypes.byref(problem._h), ctypes.byref(problem._v),
                                _ptr(problem.track_hits), problem.n_tracks, ctypes.byref(problem._p), _ptr(a),
                                int(steps), int(relinearize_every), _ptr(history), _ptr(ws), ws.numel() * 8,
                                _stream(stream)), "ut_align_solve")
    return a, history
