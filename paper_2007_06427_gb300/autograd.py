"""J(u, T) as a torch.autograd.Function whose backward is the library's adjoint kernel.

Forward: J_b = int_0^1 int_0^L r_b^2 dx ds for every loop b of a packed batch (Eq.
cost_function), computed by ``ks_residual``.  Backward: the adjoint gradient of Eq.
KS_L_dagger from ``ks_adjoint_grad``: with G = L^dag_1 r on the grid, the exact derivative of
the discrete J_b with respect to the grid values of loop b is (2 L / (Nx Ns_b)) G, and
dJ_b/dT_b = 2 L^dag_2.  The upstream gradient of each loop scales its block.

Both calls run on the GPU; tensors must live on the handle's device with the handle's element
type (float64 for FP64 / MIXED handles, float32 for FP32 handles).
"""
from __future__ import annotations

import torch

from . import ks_loop as K


class KSLoopJ(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u: torch.Tensor, T: torch.Tensor, loop: "K.KSLoop"):
        if not (u.is_cuda and T.is_cuda):
            raise ValueError("KSLoopJ needs CUDA tensors")
        u = u.contiguous()
        T = T.contiguous()
        J = torch.empty(loop.batch, dtype=torch.float64, device=u.device)
        K.ks_residual(loop.handle, u, T, None, J, torch.cuda.current_stream(u.device))
        ctx.save_for_backward(u, T)
        ctx.loop = loop
        return J

    @staticmethod
    def backward(ctx, gJ: torch.Tensor):
        u, T = ctx.saved_tensors
        loop = ctx.loop
        G = torch.empty_like(u)
        dJdT = torch.empty_like(T)
        K.ks_adjoint_grad(loop.handle, u, T, G, dJdT, torch.cuda.current_stream(u.device))
        gu = gT = None
        gJ = gJ.to(torch.float64)
        if ctx.needs_input_grad[0]:
            fac = grid_factor(loop, u.device)                       # 2 L / (Nx Ns_b) per point
            per_loop = torch.repeat_interleave(gJ, loop_sizes(loop, u.device))
            gu = G * (fac * per_loop).to(G.dtype)
        if ctx.needs_input_grad[1]:
            gT = dJdT * gJ
        return gu, gT, None


def loop_sizes(loop, device):
    key = ("sizes", str(device))
    cache = loop.__dict__.setdefault("_cache", {})
    if key not in cache:
        cache[key] = torch.tensor([n * loop.nx for n in loop.ns], dtype=torch.int64, device=device)
    return cache[key]


def grid_factor(loop, device):
    key = ("fac", str(device))
    cache = loop.__dict__.setdefault("_cache", {})
    if key not in cache:
        f = torch.tensor([2.0 * loop.L / (loop.nx * n) for n in loop.ns], dtype=torch.float64,
                         device=device)
        cache[key] = torch.repeat_interleave(f, loop_sizes(loop, device))
    return cache[key]


def cost(u: torch.Tensor, T: torch.Tensor, loop: "K.KSLoop") -> torch.Tensor:
    """J per loop, differentiable in u (packed grid values) and T."""
    return KSLoopJ.apply(u, T, loop)
