"""torch.autograd wrappers of the COLA run and of the loss-grid density (reverse mode).

Marshalling only: the forward is cola_run_checkpointed and the backward cola_adjoint /
cola_grid_density_adjoint, all in libcola.so.  The forward keeps one position snapshot per step
([n_step, 3, n] float32) for the backward, which recomputes each step's PM force from it.

    ctx = Context(Params(...))
    w = white_noise.requires_grad_()
    s, v, psi1, psi2 = cola_run(ctx, w)
    delta = grid_density(ctx, s, 64)
    ((delta - target) ** 2).sum().backward()      # w.grad = dL/dw
"""

from __future__ import annotations

import torch

from .binding import Context


class ColaRun(torch.autograd.Function):
    """(white noise [n]) -> (s, v_res, Psi1, Psi2), each [3, n] float32 in mesh cells."""

    @staticmethod
    def forward(fctx, white_noise, cola: Context):
        wn = white_noise.detach().contiguous()
        out = cola.run_checkpointed(wn)
        fctx.cola = cola
        fctx.save_for_backward(wn, out["ckpt"])
        return out["s"], out["v"], out["psi1"], out["psi2"]

    @staticmethod
    def backward(fctx, g_s, g_v, g_p1, g_p2):
        wn, ckpt = fctx.saved_tensors
        cola = fctx.cola

        def prep(g):
            return None if g is None else g.contiguous().to(torch.float32)

        g_s = prep(g_s)
        if g_s is None:
            g_s = torch.zeros((3, cola.p.n), dtype=torch.float32, device=wn.device)
        lam_w = cola.adjoint(wn, ckpt, g_s, prep(g_v), prep(g_p1), prep(g_p2))
        return lam_w, None


class GridDensity(torch.autograd.Function):
    """(s [3, n]) -> CIC density contrast [ngrid]^3 of the particles (continuous weights)."""

    @staticmethod
    def forward(fctx, s, cola: Context, ngrid: int):
        sd = s.detach().contiguous()
        fctx.cola = cola
        fctx.ngrid = int(ngrid)
        fctx.save_for_backward(sd)
        return cola.grid_density(sd, ngrid)

    @staticmethod
    def backward(fctx, g_delta):
        (sd,) = fctx.saved_tensors
        return fctx.cola.grid_density_adjoint(sd, fctx.ngrid, g_delta.contiguous().to(torch.float32)), None, None


def cola_run(cola: Context, white_noise):
    """Differentiable cola_run: returns (s, v_res, Psi1, Psi2)."""
    return ColaRun.apply(white_noise, cola)


def grid_density(cola: Context, s, ngrid: int):
    """Differentiable loss-grid density contrast of positions s."""
    return GridDensity.apply(s, cola, ngrid)
