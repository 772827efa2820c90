"""A and A^T behind torch.autograd, with gradients for the scan nonidealities.

The paper motivates a joint 3D model by the per-scan nonidealities that a
sequential pipeline cannot absorb (Sec. 1: amplifier drift, coil gain, tissue
loading). This module exposes b = A(g, w) x with per-angle gains g (the B
operator) and PSF width w (the H operator) as differentiable inputs:

    d loss / d x   = A^T grad_b                      (library adjoint)
    d loss / d g_m = <grad_b[m], A_m x |_{g_m = 1}>  (real inner product, FP64 sums)
    d loss / d w   = <grad_b, (dA/dw) x>             (PSF taps replaced by dh/dw)

Forward keeps the projections P x as the activation checkpoint (one [M, N_z, N]
tensor); backward reapplies only the line operators to it. Every product runs in
the library's CUDA kernels.
"""

import torch

from .operator import FFLOperator


class _ApplyA(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, gains, fwhm, op):
        g_host = [float(v) for v in gains.detach().cpu().reshape(-1)]
        if getattr(op, "gains", None) != g_host:
            op.set_gain(g_host)
        w = float(fwhm.detach().cpu().reshape(-1)[0])
        if w != op.fwhm:
            op.set_fwhm(w)
        proj = op.project(x.contiguous())
        b = op.line_forward(proj)
        ctx.save_for_backward(proj)
        ctx.op = op
        ctx.gshape, ctx.wshape = gains.shape, fwhm.shape
        return b

    @staticmethod
    def backward(ctx, grad_b):
        (proj,) = ctx.saved_tensors
        op = ctx.op
        gb = grad_b.contiguous().float()
        gx = None
        if ctx.needs_input_grad[0]:
            gx = op.backproject(op.line_adjoint(gb))
        gg, gw = op.param_grad_proj(proj, gb, want_gain=ctx.needs_input_grad[1], want_fwhm=ctx.needs_input_grad[2])
        gg = gg.reshape(ctx.gshape).to(torch.float32) if gg is not None else None
        gw = gw.reshape(ctx.wshape).to(torch.float32) if gw is not None else None
        return gx, gg, gw, None


def apply_a(op: FFLOperator, x, gains, fwhm):
    """b = A(gains, fwhm) x, differentiable in x, gains [M] and fwhm (1-element tensor)."""
    return _ApplyA.apply(x, gains, fwhm, op)


def calibrate(op: FFLOperator, b, x0=None, gains0=None, fwhm0=None, iters=200, lr_x=None, lr_g=1e-2, lr_w=2e-2,
              lam=0.0, fit_gain=True, fit_fwhm=True):
    """Joint volume + calibration fit: minimise 0.5 ||A(g, w) x - b||^2 (+ lam/2 ||T x||^2)
    over x >= 0, per-angle gains g and PSF width w with Adam on (g, w) and projected
    gradient steps on x. Returns (x, gains, fwhm, loss history)."""
    dev = op.device
    x = (torch.zeros(op.vol_shape, device=dev) if x0 is None else x0.clone()).requires_grad_(True)
    g = torch.tensor([1.0] * op.n_angles if gains0 is None else list(gains0), device=dev,
                     dtype=torch.float32, requires_grad=fit_gain)
    w = torch.tensor([op.fwhm if fwhm0 is None else float(fwhm0)], device=dev, dtype=torch.float32,
                     requires_grad=fit_fwhm)
    if lr_x is None:
        lr_x = 1.0 / op.power_norm(20, 1234)
    params = [p for p in (g, w) if p.requires_grad]
    opt = torch.optim.Adam([{"params": [g], "lr": lr_g}, {"params": [w], "lr": lr_w}]) if params else None
    hist = []
    for _ in range(iters):
        if opt:
            opt.zero_grad()
        if x.grad is not None:
            x.grad = None
        r = apply_a(op, x, g, w) - b
        loss = 0.5 * (r.double() ** 2).sum()
        loss.backward()
        with torch.no_grad():
            grad = x.grad
            if lam > 0:
                tx = op.apply_ttt(x.detach().contiguous())
                loss = loss + 0.5 * lam * (x.double() * tx.double()).sum()
                grad = grad + lam * tx
            hist.append(float(loss))
            x -= lr_x * grad
            x.clamp_(min=0.0)
        if opt:
            opt.step()
            with torch.no_grad():
                w.clamp_(min=0.5)
    return x.detach(), g.detach(), w.detach(), hist
