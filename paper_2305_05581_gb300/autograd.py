"""torch.autograd.Function over tns_heff_apply / tns_heff_adjoint.

Argument marshalling only: forward calls the library's H_eff*psi, backward
its adjoint (gradients with respect to the wavefunction and to the left and
right operator arenas).  The arenas are exposed as CUDA tensors that alias
the library's own device memory.
"""
from __future__ import annotations

import torch

from .binding import TNS_FP64


class _DeviceView:
    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 2}


def arena_tensor(ctx, site: int, side: int) -> torch.Tensor:
    """CUDA tensor aliasing the left (0) or right (1) operator arena of the step."""
    ptr, n = ctx.env_arena(site, side)
    return torch.as_tensor(_DeviceView(ptr, n), device="cuda")


class HeffFunction(torch.autograd.Function):
    """y = H_eff(L, R) x at one two-site step.  ``larena`` / ``rarena`` must be
    the tensors returned by :func:`arena_tensor` for this step (their values
    are read by the library; gradients are returned for them)."""

    @staticmethod
    def forward(fctx, x, larena, rarena, ctx, site):
        y = torch.empty_like(x)
        ctx.heff_apply_ptr(site, x.data_ptr(), y.data_ptr(), 1, TNS_FP64)
        fctx.save_for_backward(x)
        fctx.tns = (ctx, site, larena.numel(), rarena.numel())
        return y

    @staticmethod
    def backward(fctx, yb):
        (x,) = fctx.saved_tensors
        ctx, site, nl, nr = fctx.tns
        yb = yb.contiguous()
        xb = torch.empty_like(x)
        lb = torch.empty(nl, dtype=torch.float64, device=x.device)
        rb = torch.empty(nr, dtype=torch.float64, device=x.device)
        torch.cuda.synchronize()
        ctx.heff_adjoint_ptr(site, x.data_ptr(), yb.data_ptr(), xb.data_ptr(), lb.data_ptr(), rb.data_ptr())
        return xb, lb, rb, None, None


def heff(x, larena, rarena, ctx, site):
    return HeffFunction.apply(x, larena, rarena, ctx, site)


class IntegralEnergy(torch.autograd.Function):
    """E(h, v) = <psi| H_eff(h, v) |psi> / <psi|psi> at one two-site step with
    the MPS isometries fixed (the differentiation form's energy functional).

    forward loads (h, v) into the context, builds the step's environment and
    applies H_eff; backward returns dE/dh and dE/dv from tns_rdm (reverse mode
    through H_eff*psi and the whole renormalisation chain of both blocks,
    done natively by the library): dE/dh = gamma (symmetrised) and
    dE/dv = Gamma / 2 averaged over the eight index permutations of (ij|kl),
    the only part of dE/dv defined for integrals with that symmetry.  h and v
    are CPU float64 tensors (copied into the library); psi is a CUDA tensor
    in the step's layout."""

    @staticmethod
    def forward(fctx, h, v, psi, ctx, site):
        ctx.load_integrals(h.detach().cpu().numpy(), v.detach().cpu().numpy())
        ctx.build_env(site)
        y = torch.empty_like(psi)
        ctx.heff_apply_ptr(site, psi.data_ptr(), y.data_ptr(), 1, TNS_FP64)
        e = torch.dot(psi, y) / torch.dot(psi, psi)
        fctx.tns = (ctx, site, h.shape[0])
        fctx.save_for_backward(psi)
        return e.detach().cpu()

    @staticmethod
    def backward(fctx, ge):
        (psi,) = fctx.saved_tensors
        ctx, site, N = fctx.tns
        gamma, Gamma = ctx.rdm_ptr(site, psi.data_ptr(), N)
        g = float(ge)
        return (torch.from_numpy(g * gamma), torch.from_numpy(0.5 * g * Gamma), None, None, None)


def integral_energy(h, v, psi, ctx, site):
    return IntegralEnergy.apply(h, v, psi, ctx, site)
