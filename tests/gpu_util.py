"""Helpers for the GPU tests: run the CUDA path through the C ABI on torch
device memory, and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np
import torch

from paper_2309_08655_gb300 import rt

F64 = torch.float64


def dev():
    return torch.device("cuda:0")


def gpu_sample(star_kw: dict, u: np.ndarray):
    star = rt.Star(rt.make_params(**star_kw))
    n = u.shape[1]
    ud = torch.from_numpy(np.ascontiguousarray(u)).to(dev())
    state = torch.empty((8, n), dtype=F64, device=dev())
    w = torch.empty(n, dtype=F64, device=dev())
    st = torch.empty(n, dtype=torch.uint8, device=dev())
    code = rt.rt_sample_conversion_surface(star, n, ud, state, w, st)
    torch.cuda.synchronize()
    return star, state, w, st, code


def gpu_trace(star, state, status, **opts):
    n = state.shape[1]
    nacc = torch.zeros(n, dtype=torch.int32, device=dev())
    nrej = torch.zeros(n, dtype=torch.int32, device=dev())
    ctr = torch.zeros(8, dtype=torch.int64, device=dev())
    rt.rt_trace_forward(star, n, state, status, nacc, nrej, ctr, rt.make_opts(**opts))
    torch.cuda.synchronize()
    return nacc, nrej, ctr


def gpu_bin(star, state, w, status, nth=64, nph=32, nnu=128, nu_lo=0.0, nu_hi=9.0):
    n = state.shape[1]
    hist = torch.empty((nth, nph, nnu), dtype=F64, device=dev())
    sky = torch.empty((nth, nph), dtype=F64, device=dev())
    spec = torch.empty(nnu, dtype=F64, device=dev())
    oor = torch.empty(1, dtype=F64, device=dev())
    rt.rt_bin_spectrum(star, n, state, w, status, nth, nph, nnu, nu_lo, nu_hi, hist, sky, spec,
                       oor)
    torch.cuda.synchronize()
    return hist.cpu().numpy(), sky.cpu().numpy(), spec.cpu().numpy(), float(oor.cpu()[0])


def to_np(*ts):
    return [t.cpu().numpy() for t in ts]


def rel_state_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-ray max of |dx|/|x| and |dk|/|k| (state rows 0-5)."""
    dx = np.linalg.norm(a[:3] - b[:3], axis=0) / np.maximum(np.linalg.norm(b[:3], axis=0), 1e-300)
    dk = np.linalg.norm(a[3:6] - b[3:6], axis=0) / np.maximum(np.linalg.norm(b[3:6], axis=0),
                                                              1e-300)
    return np.maximum(dx, dk)


def perturbed(state0, eps, seed):
    rng = np.random.default_rng(seed)
    p = state0.copy()
    p[:6] *= 1.0 + eps * rng.standard_normal(p[:6].shape)
    return p


def well_conditioned(oracle, star_vec, state0, status0, rtol, spread_max=1e-12, **kw):
    """Oracle end states at rtol (strict FP64 build) and the spread between the
    strict build and the same source compiled with FMA contraction -- two
    equally valid FP64 evaluations.  Many production rays are produced near a
    reflection or scatter between the plasma walls of the magnetosphere and
    amplify rounding by orders of magnitude; agreement at the 1e-10 level is
    only defined for rays whose end point is insensitive to rounding (spread
    <= spread_max).  Returns (end states, statuses, well-conditioned mask,
    spread)."""
    a = state0.copy()
    sa = status0.copy()
    oracle.trace_forward(star_vec, oracle.trace_opts(rtol=rtol, **kw), a, sa)
    b = state0.copy()
    sb = status0.copy()
    oracle.trace_forward(star_vec, oracle.trace_opts(rtol=rtol, **kw), b, sb,
                         variant="contracted")
    spread = rel_state_diff(b, a)
    good = (sa == sb) & (spread <= spread_max)
    return a, sa, good, spread
