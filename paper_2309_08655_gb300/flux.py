"""Differentiable line flux: a ``torch.autograd.Function`` over the C ABI.

``line_flux(params, base, uniforms, kappa)`` samples the conversion surface
with the given uniforms, traces every ray (FP64) and returns the von
Mises-Fisher-smoothed line flux F toward the observer (rt_flux_value).  Its
backward pass calls rt_flux_gradient, the reverse-mode adjoint through the
integrator over a full step tape in device memory (checkpoints every 32 steps
when the tape does not fit); ``grad_precision`` sets the backward sweep's
arithmetic over the same FP64 replay: "fp64", "mixed" (FP64 adjoint, FP32
tangents of the ray equations' constants) or "df" (double-float).  ``params`` is a float64 tensor
(m_a [eV], B0 [G], theta_m [rad], M [Msun], R [km], inclination [rad]);
``base`` holds the other star parameters (``rt.make_params`` keywords).
Every step runs in the CUDA library; torch supplies device memory and the
autograd plumbing.
"""
from __future__ import annotations

import torch

from . import rt

PARAM_NAMES = ("m_a_eV", "B0_G", "theta_m", "M_sun", "R_km", "incl")
_GRAD_PREC = {"fp64": rt.PREC_FP64, "df": rt.PREC_DF, "mixed": rt.PREC_MIXED}


def _star(params: torch.Tensor, base: dict) -> tuple[rt.Star, float]:
    p = [float(v) for v in params.detach().cpu().tolist()]
    kw = dict(base)
    kw.update(m_a_eV=p[0], B0_G=p[1], theta_m=p[2], M_sun=p[3], R_km=p[4])
    return rt.Star(rt.make_params(**kw)), p[5]


def flux_forward(params, base, uniforms, kappa, rtol=1e-10):
    """F and the per-ray accepted step counts (no autograd)."""
    star, incl = _star(params, base)
    n = uniforms.shape[1]
    dev = uniforms.device
    f64 = torch.float64
    st = torch.empty((rt.STATE_ROWS, n), dtype=f64, device=dev)
    w = torch.empty(n, dtype=f64, device=dev)
    s = torch.empty(n, dtype=torch.uint8, device=dev)
    rt.rt_sample_conversion_surface(star, n, uniforms, st, w, s)
    nacc = torch.zeros(n, dtype=torch.int32, device=dev)
    opts = rt.make_opts(rtol=rtol, precision=rt.PREC_FP64)
    rt.rt_trace_forward(star, n, st, s, nacc, None, None, opts)
    F_ray = torch.empty(n, dtype=f64, device=dev)
    F = torch.empty(1, dtype=f64, device=dev)
    rt.rt_flux_value(star, n, st, w, s, incl, kappa, F_ray, F)
    return F, nacc, star, incl, opts


class LineFlux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, base, uniforms, kappa, rtol, grad_precision):
        F, nacc, star, incl, opts = flux_forward(params, base, uniforms, kappa, rtol)
        ctx.save_for_backward(uniforms, nacc)
        ctx.star, ctx.incl, ctx.kappa = star, incl, kappa
        ctx.opts = rt.make_opts(rtol=rtol, precision=_GRAD_PREC[grad_precision])
        return F[0].to(params.device)

    @staticmethod
    def backward(ctx, gF):
        uniforms, nacc = ctx.saved_tensors
        dev = uniforms.device
        grad = torch.empty(len(PARAM_NAMES), dtype=torch.float64, device=dev)
        F = torch.empty(1, dtype=torch.float64, device=dev)
        rt.rt_flux_gradient(ctx.star, uniforms.shape[1], uniforms, nacc, ctx.incl, ctx.kappa,
                            grad, F, opts=ctx.opts)
        return (grad.to(gF.device) * gF), None, None, None, None, None


def line_flux(params: torch.Tensor, base: dict, uniforms: torch.Tensor, kappa: float,
              rtol: float = 1e-10, grad_precision: str = "fp64") -> torch.Tensor:
    if grad_precision not in _GRAD_PREC:
        raise ValueError(f"grad_precision must be one of {sorted(_GRAD_PREC)}")
    return LineFlux.apply(params, base, uniforms, kappa, rtol, grad_precision)
