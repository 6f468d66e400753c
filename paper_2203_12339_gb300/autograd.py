"""torch.autograd wrappers: material -> coefficients -> relit shading, with
hand-written adjoints running in libtsr (Section 2.2 projection, Section 4
rendering Steps 3-5).

    B = relight(S, project(sigma_a, sigma_s', eta), l)
    B_view = (1/pi) F_t(eta, n_o . w_o) B          (optional, Eq. 6)

Gradients flow to sigma_a, sigma_s', eta (through the FP64 analytic
derivative of the dipole R_d, and through dF_t/deta of the view factor) and
to the light coefficients l.
"""
from __future__ import annotations

import torch

from . import tsr


class ProjectMaterialFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma_a, sigma_s, eta, basis):
        _, g32, _ = tsr.project_material(basis, sigma_a.detach(), sigma_s.detach(), eta.detach())
        ctx.basis = basis
        ctx.save_for_backward(sigma_a.detach(), sigma_s.detach(), eta.detach())
        return g32

    @staticmethod
    def backward(ctx, dg):
        sa, ss, et = ctx.saved_tensors
        dsa, dss, de = tsr.project_material_backward(ctx.basis, sa, ss, et, dg.contiguous())
        return dsa.to(sa.dtype), dss.to(ss.dtype), de.to(et.dtype), None


class RelightFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, light, comp):
        B = tsr.relight(comp, g.detach(), light.detach())
        ctx.comp = comp
        ctx.save_for_backward(g.detach(), light.detach())
        return B

    @staticmethod
    def backward(ctx, dB):
        g, light = ctx.saved_tensors
        dg, dl = tsr.relight_backward(ctx.comp, g, light, dB.contiguous())
        return dg, dl, None


class FresnelOutputFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, B, eta, cos_o):
        ctx.save_for_backward(B.detach(), eta.detach(), cos_o.detach())
        return tsr.fresnel_output(B.detach(), eta.detach(), cos_o.detach())

    @staticmethod
    def backward(ctx, dBout):
        B, eta, cos_o = ctx.saved_tensors
        dB, deta = tsr.fresnel_output_backward(B, eta, cos_o, dBout.contiguous())
        return dB, deta.to(eta.dtype), None


def render(comp: "tsr.Compressed", basis: "tsr.Basis", sigma_a: torch.Tensor, sigma_s: torch.Tensor,
           eta: torch.Tensor, light: torch.Tensor, cos_o: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable relight B [E][3][N] of materials (sigma_a, sigma_s' [E][3] FP64, eta [E] FP64) under
    light [J]; with cos_o [N] (n_o . w_o per vertex) the view-dependent Fresnel factor of Eq. 6 is applied."""
    g = ProjectMaterialFn.apply(sigma_a, sigma_s, eta, basis)
    B = RelightFn.apply(g, light, comp)
    if cos_o is not None:
        B = FresnelOutputFn.apply(B, eta, cos_o)
    return B
