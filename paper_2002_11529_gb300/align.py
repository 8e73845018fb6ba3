"""Detector alignment through the library's chi2 adjoint kernels.

The p-kick fit's chi2 (Sec. III-C) of tracks with fixed selected hits, as a
function of the track states theta [T,3] = (x, tx, qop) and the per-sector
alignment [4S,3] = (dx, dz, gamma), is exposed as a torch.autograd.Function
whose backward is the library's hand-written adjoint (ut_align_chi2).

solve_alignment estimates the alignment by preconditioned conjugate
gradients on the reduced Gauss-Newton system (track states profiled out by
a refit): every step is one reduced Hessian-vector product (ut_align_hvp),
the preconditioner the per-sector 3x3 Gauss-Newton blocks.  The detector
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


def _block_inverse(h6: torch.Tensor) -> torch.Tensor:
    """Inverse of the per-sector symmetric 3x3 blocks [a b c; b d e; c e f]
    (h6 = a, b, c, d, e, f) by cofactors in double; zero for sectors without
    hits (a == 0) or a singular block.  Returns [4S, 3, 3]."""
    h = h6.to(torch.float64)
    a, b, c, d, e, f = (h[:, i] for i in range(6))
    A = d * f - e * e
    Bc = c * e - b * f
    C = b * e - c * d
    D = a * f - c * c
    E = b * c - a * e
    F = a * d - b * b
    det = a * A + b * Bc + c * C
    ok = (a > 0) & (det != 0)
    r = torch.where(ok, 1.0 / torch.where(ok, det, torch.ones_like(det)), torch.zeros_like(det))
    inv = torch.stack([torch.stack([A, Bc, C], -1), torch.stack([Bc, D, E], -1), torch.stack([C, E, F], -1)], -2)
    return inv * r[:, None, None]


def solve_alignment(problem: AlignmentProblem, steps: int = 20, relinearize_every: int = 10,
                    align0: torch.Tensor | None = None):
    """Estimate the alignment in `steps` preconditioned CG steps (one reduced
    Hessian-vector product each), re-linearising (refit + new gradient)
    every `relinearize_every` steps.  Returns (align, history)."""
    dev = problem.track_hits.device
    a = torch.zeros((4 * problem.S, 3), dtype=torch.float32, device=dev) if align0 is None else align0.clone()
    history = []
    done = 0
    while done < steps:
        theta = problem.refit(a)
        c2, _, g, hblk = problem.chi2(theta, a, grads=True)
        history.append(float(c2.item()))
        Minv = _block_inverse(hblk)
        apply_m = lambda r: torch.einsum("sij,sj->si", Minv, r)
        x = torch.zeros((4 * problem.S, 3), dtype=torch.float64, device=dev)
        r = -g.to(torch.float64)
        z = apply_m(r)
        p = z.clone()
        rz = (r * z).sum()
        for _ in range(min(relinearize_every, steps - done)):
            Ap = problem.hvp(theta, a, p)
            pAp = (p * Ap).sum()
            if not torch.isfinite(pAp) or pAp <= 0:
                break
            alpha = rz / pAp
            x += alpha * p
            r -= alpha * Ap
            z = apply_m(r)
            rz_new = (r * z).sum()
            p = z + (rz_new / rz) * p
            rz = rz_new
            done += 1
        else:
            a = a + x.to(torch.float32)
            continue
        a = a + x.to(torch.float32)
        break
    theta = problem.refit(a)
    history.append(float(problem.chi2(theta, a)[0].item()))
    return a, history
